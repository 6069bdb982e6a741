// Tensor-core (tcgen05) path of Eq. 19: every mode product runs as 128-row
// tiles of pencils (M) against the zero-padded n x n eigenvector block (K = N =
// n rounded up to 16) held in shared memory, accumulating in TMEM.
//
// Precision (KX_F16X3): both operands are split into fp16 hi + lo halves after
// scaling by a power of two (2^14 for V, |V| <= 1; per item for the data), and
// D = A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in fp32.  Each half has
// 11 significant bits, so the product keeps ~22 bits; the power-of-two scales
// are undone exactly in the epilogue.
//
// Passes over a chunk of items (pair products or caller vectors), all in the
// natural grid layout (x1 fastest) of fp32 scratch:
//   X3F  rho = psi_i psi_j (prologue), contract x3 with V3   [A MN-major]
//   X2F  contract x2 with V2                                  [A MN-major]
//   X1   contract x1 with V1, scale by f(Lambda) (+ Parseval energy), contract
//        back with V1^T                                       [A K-major]
//   X2I  contract k2 with V2^T                                [A MN-major]
//   X3I  contract k3 with V3^T, write phi (pair mode) or f(L)b (vector mode)
// then acc_kernel adds g_j psi_j phi_ij and g_i psi_i phi_ij into the fp32
// accumulators, one thread per four grid points, group by group.
//
// Each pass kernel is persistent (one CTA per SM) and warp-specialised:
//   warps 0-7   epilogue (TMEM lane quadrant = warp % 4, column half = warp / 4)
//   warps 8-15  producers: global fp32 -> scale -> fp16 hi/lo -> shared stage
//   warp 16     TMEM allocation and MMA issue (one thread)
// with an S-deep ring of shared A stages and two TMEM accumulator slots, so
// loads, MMAs and stores of consecutive tiles overlap.
#include "kx_internal.h"
#include "kx_tc_ptx.cuh"

#include <algorithm>
#include <cmath>
#include <string>

namespace kx {
namespace {

enum PassKind { P_X3F = 0, P_X2F = 1, P_X1 = 2, P_X2I = 3, P_X3I = 4 };

constexpr int kEpiWarps = 8;
constexpr int kProdWarps = 8;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kProdThreads = 32 * kProdWarps;
constexpr int kMmaWarp = kEpiWarps + kProdWarps;
constexpr int kThreads = 32 * (kEpiWarps + kProdWarps + 1);
constexpr int kMaxStages = 4;
constexpr int kProdUnroll = 3;
constexpr size_t kSmemBudget = 225 * 1024;

struct PassArgs {
    int n1, n2, n3;
    int nc;                // contraction length of this pass
    int np;                // nc rounded up to 16 (MMA K and N)
    int stages;            // shared A stages in the ring
    long long rows_pp;     // rows (pencils) per item
    long long total_rows;  // items * rows_pp
    long long N;
    const float *in;
    float *out;
    const __half *Vs;      // [2][np*np]: hi block, lo block (8x8 core-matrix order)
    const int2 *pairs;     // pair mode: (i, j) of each item of the chunk
    const float *psi32;    // [n_orb][N]
    const float *orb_max;  // [n_orb] max |psi|
    const float *src_max;  // vector mode: per-item max |b|
    int rhs_mode;
    const float *in_max;   // per-item max |input| (passes after X3F)
    float *out_max;        // per-item max |output| (nullable)
    const float *f32;      // f(Lambda), natural layout
    float mid_bound;       // fmax * sqrt(n1)
    double *e_partial;     // per-CTA energy partial (nullable)
    int energy_only;
    const double *occ;
    double *xout;          // vector mode output of X3I (fp64)
    int *status;
    long long timeout_cycles;
};

__device__ __forceinline__ int scale_exp(float mx) {
    // e such that mx * 2^e < 2^14 (mx = m 2^k, m in [0.5, 1)  =>  e = 14 - k)
    int k = 0;
    if (mx > 0.f && isfinite(mx)) frexpf(mx, &k);
    return 14 - k;
}

__device__ __forceinline__ void split8(const float *v, uint4 &hi, uint4 &lo) {
    __half2 h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __half2 hh = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
        float2 hf = __half22float2(hh);
        h[i] = hh;
        l[i] = __floats2half2_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
    }
    hi = *reinterpret_cast<uint4 *>(h);
    lo = *reinterpret_cast<uint4 *>(l);
}

__device__ __forceinline__ void ld8(const float *p, float *v) {
    float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

template <int PASS>
__device__ __forceinline__ float item_in_max(const PassArgs &a, long long item) {
    if (PASS == P_X3F) {
        if (a.rhs_mode) return a.src_max[item];
        int2 ij = a.pairs[item];
        return a.orb_max[ij.x] * a.orb_max[ij.y];
    }
    return a.in_max[item];
}

// Source address of task t (8 consecutive fp32 values) of a tile and its
// shared-memory offset; returns false for padding (zero) tasks.  Pair mode of
// X3F has two sources (psi_i, psi_j).
template <int PASS>
__device__ __forceinline__ bool task_src(const PassArgs &a, long long tile, int t, const float *&p0,
                                         const float *&p1, float &scale, int &soff) {
    const int kp = a.np;
    const long long n12 = (long long)a.n1 * a.n2;
    if (PASS == P_X1) {
        // K-major: element (m, k) at (m/8)*(kp*16) + (k/8)*128 + (m%8)*16 + (k%8)*2
        const int nkc = kp >> 3;
        const int mi = t & 7;
        const int kc = (t >> 3) % nkc;
        const int mg = (t >> 3) / nkc;
        soff = mg * (kp * 16) + kc * 128 + mi * 16;
        const long long R = tile * 128 + mg * 8 + mi;
        if (R >= a.total_rows || kc * 8 >= a.nc) return false;
        const long long item = R / a.rows_pp, local = R % a.rows_pp;
        p0 = a.in + item * a.N + local * a.n1 + kc * 8;
        p1 = nullptr;
        scale = ldexpf(1.f, scale_exp(item_in_max<PASS>(a, item)));
        return true;
    } else {
        // MN-major: element (m, k) at (m/8)*128 + (k/8)*2048 + (k%8)*16 + (m%8)*2
        const int ki = t & 7;
        const int g = (t >> 3) & 15;
        const int kg = t >> 7;
        const int k = kg * 8 + ki;
        soff = g * 128 + kg * 2048 + ki * 16;
        const long long R0 = tile * 128 + g * 8;
        if (R0 >= a.total_rows || k >= a.nc) return false;
        const long long item = R0 / a.rows_pp, local = R0 % a.rows_pp;
        scale = ldexpf(1.f, scale_exp(item_in_max<PASS>(a, item)));
        p1 = nullptr;
        if (PASS == P_X3F) {
            const long long x = (long long)k * n12 + local;  // (x3 = k, position = local)
            if (a.rhs_mode) {
                p0 = a.in + item * a.N + x;
            } else {
                const int2 ij = a.pairs[item];
                p0 = a.psi32 + (long long)ij.x * a.N + x;
                p1 = a.psi32 + (long long)ij.y * a.N + x;
            }
        } else if (PASS == P_X2F || PASS == P_X2I) {
            const long long k3 = local / a.n1, x1 = local % a.n1;  // rows (k3, x1)
            p0 = a.in + item * a.N + k3 * n12 + (long long)k * a.n1 + x1;
        } else {  // P_X3I: rows = positions, K = k3
            p0 = a.in + item * a.N + (long long)k * n12 + local;
        }
        return true;
    }
}

// Producer side: stage one 128-row tile of the A operand (scaled, split).
// The loads of kProdUnroll tasks are issued before any of them is converted.
template <int PASS>
__device__ __forceinline__ void produce_tile(const PassArgs &a, long long tile, uint8_t *Ahi, uint8_t *Alo,
                                             int ptid) {
    const int ntask = (PASS == P_X1) ? 128 * (a.np >> 3) : 16 * a.np;
    const bool two = (PASS == P_X3F) && !a.rhs_mode;
    for (int t0 = ptid; t0 < ntask; t0 += kProdThreads * kProdUnroll) {
        float v[kProdUnroll][8], u[kProdUnroll][8];
        float sc[kProdUnroll];
        int off[kProdUnroll];
        bool ok[kProdUnroll];
#pragma unroll
        for (int r = 0; r < kProdUnroll; ++r) {
            const int t = t0 + r * kProdThreads;
            const float *p0 = nullptr, *p1 = nullptr;
            ok[r] = false;
            off[r] = -1;
            sc[r] = 0.f;
            if (t < ntask) ok[r] = task_src<PASS>(a, tile, t, p0, p1, sc[r], off[r]);
            if (ok[r]) {
                ld8(p0, v[r]);
                if (two) ld8(p1, u[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < kProdUnroll; ++r) {
            if (off[r] < 0) continue;
            float w[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                float x = ok[r] ? v[r][c] : 0.f;
                if (two && ok[r]) x *= u[r][c];
                w[c] = x * sc[r];
            }
            uint4 hi, lo;
            split8(w, hi, lo);
            *reinterpret_cast<uint4 *>(Ahi + off[r]) = hi;
            *reinterpret_cast<uint4 *>(Alo + off[r]) = lo;
        }
    }
}

// D = A_hi B_hi + A_hi B_lo + A_lo B_hi over K = np (single issuing thread).
// The tensor core rounds its fp32 accumulator toward zero at every instruction,
// so a long chain of large partial sums drifts low.  To keep that drift small
// the two small cross products are issued first into accumulator Da, and the
// hi*hi chain is split over Da (even k-steps) and Db (odd k-steps); the
// epilogue adds Da + Db with round-to-nearest.
__device__ __forceinline__ void issue_split_mma(uint32_t tmem_a, uint32_t tmem_b, uint32_t a_hi, uint32_t a_lo,
                                                bool a_kmajor, uint32_t v_hi, uint32_t v_lo, bool inverse, int np) {
    const uint32_t idesc = ptx::idesc_f16(128, np, a_kmajor ? 0 : 1, inverse ? 0 : 1);
    const uint32_t a_lbo = a_kmajor ? 128u : 2048u;
    const uint32_t a_sbo = a_kmajor ? (uint32_t)(np * 16) : 128u;
    const uint32_t a_step = a_kmajor ? 256u : 4096u;
    // V stored as 8x8 core matrices, row block of 8 x-rows = np*16 bytes.
    //   forward  (B[x][k] = V[x][k]): MN-major, K (=x) stride np*16, N (=k) stride 128
    //   inverse  (B[k][x] = V[x][k]): K-major,  K (=k) stride 128,   N (=x) stride np*16
    const uint32_t b_lbo = inverse ? 128u : (uint32_t)(np * 16);
    const uint32_t b_sbo = inverse ? (uint32_t)(np * 16) : 128u;
    const uint32_t b_step = inverse ? 256u : (uint32_t)(np * 32);
    const int nks = np >> 4;
    for (int ks = 0; ks < nks; ++ks) {
        const uint64_t ah = ptx::sdesc(a_hi + ks * a_step, a_lbo, a_sbo);
        const uint64_t al = ptx::sdesc(a_lo + ks * a_step, a_lbo, a_sbo);
        const uint64_t bh = ptx::sdesc(v_hi + ks * b_step, b_lbo, b_sbo);
        const uint64_t bl = ptx::sdesc(v_lo + ks * b_step, b_lbo, b_sbo);
        ptx::mma_f16(tmem_a, ah, bl, idesc, ks > 0 ? 1u : 0u);
        ptx::mma_f16(tmem_a, al, bh, idesc, 1u);
    }
    for (int ks = 0; ks < nks; ++ks) {
        const uint64_t ah = ptx::sdesc(a_hi + ks * a_step, a_lbo, a_sbo);
        const uint64_t bh = ptx::sdesc(v_hi + ks * b_step, b_lbo, b_sbo);
        if (ks & 1)
            ptx::mma_f16(tmem_b, ah, bh, idesc, ks > 1 ? 1u : 0u);
        else
            ptx::mma_f16(tmem_a, ah, bh, idesc, 1u);
    }
}

// Da + Db for 16 columns of this thread's lane (Db is empty when K = 16).
__device__ __forceinline__ void tmem_ld16_sum(uint32_t ta, uint32_t tb, bool two, float *v) {
    ptx::tmem_ld16(ta, v);
    if (two) {
        float w[16];
        ptx::tmem_ld16(tb, w);
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] += w[c];
    }
}

// Bounded wait shared by all roles: gives up when the limit elapses or another
// role already gave up (then every role leaves its loop and the CTA exits).
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, const PassArgs &a, volatile int *abort) {
    const long long t0 = clock64();
    while (!ptx::mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > a.timeout_cycles) {
            *abort = 1;
            atomicExch(a.status, KX_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// Warp-uniform form for roles that follow the wait with warp-collective
// instructions (tcgen05.ld): every lane sees the same outcome.
__device__ __forceinline__ bool wait_bar_warp(uint64_t *bar, uint32_t parity, const PassArgs &a,
                                              volatile int *abort) {
    const bool ok = wait_bar(bar, parity, a, abort);
    return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ void track_max(float *out_max, long long item, float m, bool valid) {
    if (out_max == nullptr) return;
    const long long item0 = __shfl_sync(0xffffffffu, item, 0);
    const bool same = __all_sync(0xffffffffu, !valid || item == item0);
    if (same) {
        float r = valid ? m : 0.f;
        for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
        if ((threadIdx.x & 31) == 0 && r > 0.f) atomicMax(reinterpret_cast<int *>(out_max + item0), __float_as_int(r));
    } else if (valid && m > 0.f) {
        atomicMax(reinterpret_cast<int *>(out_max + item), __float_as_int(m));
    }
}

struct Bars {
    uint64_t full[kMaxStages];
    uint64_t empty[kMaxStages];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t tfull2[2];
    uint64_t mid_full;
    uint64_t mid_empty;
    uint64_t drain;
};

template <int PASS>
__global__ void __launch_bounds__(kThreads, 1) tc_pass_kernel(const PassArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int np = a.np;
    const int S = a.stages;
    const size_t stage_bytes = (size_t)2 * 128 * np * 2;  // hi + lo
    uint8_t *Vhi = smem;
    uint8_t *Vlo = Vhi + np * np * 2;
    uint8_t *stage0 = Vlo + np * np * 2;
    uint8_t *mid = stage0 + S * stage_bytes;  // X1 only
    __shared__ Bars bars;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    __shared__ double s_red[kEpiWarps];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool with_inv = (PASS == P_X1) && !a.energy_only;
    const uint32_t tcols = (4 * np <= 256) ? 256u : 512u;
    if (warp == kMmaWarp) {
        ptx::tmem_alloc(&tmem_slot, tcols);
        ptx::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            ptx::mbar_init(&bars.full[s], kProdThreads);
            ptx::mbar_init(&bars.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&bars.tfull[b], 1);
            ptx::mbar_init(&bars.tempty[b], kEpiThreads);
            ptx::mbar_init(&bars.tfull2[b], 1);
        }
        ptx::mbar_init(&bars.mid_full, kEpiThreads);
        ptx::mbar_init(&bars.mid_empty, 1);
        ptx::mbar_init(&bars.drain, 1);
        ptx::fence_mbar_init();
        s_abort = 0;
    }
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.Vs);
        uint4 *dst = reinterpret_cast<uint4 *>(Vhi);
        const int n16 = (2 * np * np * 2) / 16;
        for (int i = tid; i < n16; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    ptx::fence_proxy_async_smem();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const long long n_tiles = (a.total_rows + 127) / 128;
    const int n_my = (int)((n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);  // tiles of this CTA
    const long long n12 = (long long)a.n1 * a.n2;
    const bool two_acc = (np >> 4) > 1;

    if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t sVhi = ptx::smem_u32(Vhi), sVlo = ptx::smem_u32(Vlo);
            const bool inv = (PASS == P_X2I || PASS == P_X3I);
            bool ok = true;
            for (int it = 0; it <= n_my && ok; ++it) {
                if (it < n_my) {
                    const int s = it % S, b = it & 1;
                    ok = wait_bar(&bars.full[s], (uint32_t)((it / S) & 1), a, &s_abort);
                    if (ok && it >= 2) ok = wait_bar(&bars.tempty[b], (uint32_t)(((it >> 1) - 1) & 1), a, &s_abort);
                    if (!ok) break;
                    ptx::tc_fence_after();
                    const uint32_t sA = ptx::smem_u32(stage0 + s * stage_bytes);
                    const uint32_t da = tmem + (uint32_t)(b * 2 * np);
                    issue_split_mma(da, da + (uint32_t)np, sA, sA + (uint32_t)(128 * np * 2), PASS == P_X1, sVhi,
                                    sVlo, inv, np);
                    ptx::mma_commit(&bars.empty[s]);
                    ptx::mma_commit(&bars.tfull[b]);
                }
                if (with_inv && it >= 1) {
                    const int j = it - 1, b = j & 1;
                    ok = wait_bar(&bars.mid_full, (uint32_t)(j & 1), a, &s_abort);
                    if (!ok) break;
                    ptx::tc_fence_after();
                    const uint32_t sM = ptx::smem_u32(mid);
                    const uint32_t da = tmem + (uint32_t)(b * 2 * np);
                    issue_split_mma(da, da + (uint32_t)np, sM, sM + (uint32_t)(128 * np * 2), true, sVhi, sVlo, true,
                                    np);
                    ptx::mma_commit(&bars.mid_empty);
                    ptx::mma_commit(&bars.tfull2[b]);
                }
            }
            if (!ok) {
                // a wait gave up: one more bounded wait for the MMAs already issued
                ptx::mma_commit(&bars.drain);
                ptx::mbar_wait_bounded(&bars.drain, 0, a.timeout_cycles);
            }
        }
        __syncwarp();
    } else if (warp >= kEpiWarps) {
        // ------------------------------------------------------------ producers
        const int ptid = tid - kEpiThreads;
        for (int it = 0; it < n_my; ++it) {
            const int s = it % S;
            if (it >= S && !wait_bar(&bars.empty[s], (uint32_t)(((it / S) - 1) & 1), a, &s_abort)) break;
            if (s_abort) break;
            uint8_t *Ahi = stage0 + s * stage_bytes;
            produce_tile<PASS>(a, blockIdx.x + (long long)it * gridDim.x, Ahi, Ahi + 128 * np * 2, ptid);
            ptx::fence_proxy_async_smem();
            ptx::mbar_arrive(&bars.full[s]);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3, half = warp >> 2;
        const int m = 32 * q + lane;  // TMEM lane == tile row of this thread
        const int nch = np >> 4;      // 16-column chunks
        double e_acc = 0.0;
        for (int it = 0; it < n_my; ++it) {
            const int b = it & 1;
            if (!wait_bar_warp(&bars.tfull[b], (uint32_t)((it >> 1) & 1), a, &s_abort)) break;
            ptx::tc_fence_after();
            const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * 2 * np);
            const uint32_t tb = ta + (uint32_t)np;
            const long long tile = blockIdx.x + (long long)it * gridDim.x;
            const long long R = tile * 128 + m;
            const bool valid = R < a.total_rows;
            const long long item = valid ? R / a.rows_pp : 0;
            const long long local = valid ? R % a.rows_pp : 0;
            const float in_mx = valid ? item_in_max<PASS>(a, item) : 0.f;
            const float unscale = ldexpf(1.f, -(scale_exp(in_mx) + kVScaleExp));
            float my_max = 0.f;

            if (PASS == P_X1) {
                const int e_mid = scale_exp(a.mid_bound * in_mx);
                const float s_mid = ldexpf(1.f, e_mid);
                double w = 0.0;
                if (valid && a.e_partial != nullptr && !a.rhs_mode) {
                    int2 ij = a.pairs[item];
                    w = (ij.x == ij.y) ? 1.0 : 2.0;
                    if (a.occ) w *= a.occ[ij.x] * a.occ[ij.y];
                }
                if (with_inv && it >= 1 && !wait_bar_warp(&bars.mid_empty, (uint32_t)((it - 1) & 1), a, &s_abort))
                    break;
                float e_row = 0.f;
                for (int c = half; c < nch; c += 2) {
                    float v[16];
                    tmem_ld16_sum(ta + 16 * c, tb + 16 * c, two_acc, v);
                    float fk[16];
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {  // nc is a multiple of 8: each 8-column half is in or out
                        if (valid && 16 * c + 8 * h2 < a.nc) {
                            ld8(a.f32 + local * a.n1 + 16 * c + 8 * h2, fk + 8 * h2);
                        } else {
#pragma unroll
                            for (int k = 0; k < 8; ++k) fk[8 * h2 + k] = 0.f;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const float y = v[k] * unscale;
                        e_row = fmaf(fk[k] * y, y, e_row);
                        v[k] = fk[k] * y * s_mid;
                    }
                    if (with_inv) {
#pragma unroll
                        for (int h2 = 0; h2 < 2; ++h2) {
                            uint4 hi, lo;
                            split8(v + 8 * h2, hi, lo);
                            const int off = (m >> 3) * (np * 16) + (2 * c + h2) * 128 + (m & 7) * 16;
                            *reinterpret_cast<uint4 *>(mid + off) = hi;
                            *reinterpret_cast<uint4 *>(mid + 128 * np * 2 + off) = lo;
                        }
                    }
                }
                e_acc += w * (double)e_row;
                if (with_inv) {
                    ptx::fence_proxy_async_smem();
                    ptx::tc_fence_before();
                    ptx::mbar_arrive(&bars.mid_full);
                    if (!wait_bar_warp(&bars.tfull2[b], (uint32_t)((it >> 1) & 1), a, &s_abort)) break;
                    ptx::tc_fence_after();
                    const float unscale2 = ldexpf(1.f, -(e_mid + kVScaleExp));
                    for (int c = half; c < nch; c += 2) {
                        float v[16];
                        tmem_ld16_sum(ta + 16 * c, tb + 16 * c, two_acc, v);
#pragma unroll
                        for (int h2 = 0; h2 < 2; ++h2) {  // store each 8-column half that lies inside the row
                            if (!valid || 16 * c + 8 * h2 >= a.nc) continue;
                            float *w = v + 8 * h2;
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                w[k] *= unscale2;
                                my_max = fmaxf(my_max, fabsf(w[k]));
                            }
                            float4 *dst = reinterpret_cast<float4 *>(a.out + item * a.N + local * a.n1 + 16 * c + 8 * h2);
                            dst[0] = make_float4(w[0], w[1], w[2], w[3]);
                            dst[1] = make_float4(w[4], w[5], w[6], w[7]);
                        }
                    }
                    track_max(a.out_max, item, my_max, valid);
                }
            } else {
                // transposed write: one column per store, consecutive lanes = consecutive rows
                for (int c = half; c < nch; c += 2) {
                    float v[16];
                    tmem_ld16_sum(ta + 16 * c, tb + 16 * c, two_acc, v);
                    if (!valid) continue;
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int col = 16 * c + k;
                        if (col >= a.nc) break;
                        const float y = v[k] * unscale;
                        long long dst;
                        if (PASS == P_X3F || PASS == P_X3I) {
                            dst = (long long)col * n12 + local;  // [k3 or x3][position]
                        } else {
                            const long long k3 = local / a.n1, x1 = local % a.n1;
                            dst = k3 * n12 + (long long)col * a.n1 + x1;  // [k3][k2 or x2][x1]
                        }
                        if (PASS == P_X3I && a.rhs_mode) {
                            a.xout[item * a.N + dst] = (double)y;
                        } else {
                            my_max = fmaxf(my_max, fabsf(y));
                            a.out[item * a.N + dst] = y;
                        }
                    }
                }
                track_max(a.out_max, item, my_max, valid);
            }
            ptx::tc_fence_before();
            ptx::mbar_arrive(&bars.tempty[b]);
        }
        if (a.e_partial != nullptr) {
            double e = e_acc;
            for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
            if (lane == 0) s_red[warp] = e;
            ptx::named_bar(1, kEpiThreads);
            if (tid == 0) {
                double sum = 0.0;
                for (int w = 0; w < kEpiWarps; ++w) sum += s_red[w];
                a.e_partial[blockIdx.x] = sum;
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, tcols);
    }
}

// Accumulation of one chunk, group by group: one thread per four grid points
// keeps psi and the partial sums of the group's (<= kGroupSlots) orbitals in
// shared memory and visits the group's items in order, adding
// g_j psi_j phi_ij to orbital i and g_i psi_i phi_ij to orbital j; at the end
// of the group it adds the partial sums into the fp32 accumulators.  Every
// accumulator element is owned by one thread per launch and chunks run in a
// fixed order, so the result is deterministic.
constexpr int kAccThreads = 128;

__global__ void __launch_bounds__(kAccThreads) acc_kernel(const float *__restrict__ phi, const Group *__restrict__ groups,
                                                         int g0, int g1, int item0, const int2 *__restrict__ item_slot,
                                                         const float *__restrict__ psi32, const double *__restrict__ occ,
                                                         float *__restrict__ acc, long long N) {
    __shared__ float4 ps[kGroupSlots][kAccThreads];
    __shared__ float4 as[kGroupSlots][kAccThreads];
    __shared__ Group G;
    __shared__ float gs[kGroupSlots];
    const int tid = threadIdx.x;
    const long long N4 = N >> 2;
    const long long x4 = (long long)blockIdx.x * kAccThreads + tid;
    const bool valid = x4 < N4;
    const float4 *phi4 = reinterpret_cast<const float4 *>(phi);
    const float4 *psi4 = reinterpret_cast<const float4 *>(psi32);
    float4 *acc4 = reinterpret_cast<float4 *>(acc);
    for (int g = g0; g < g1; ++g) {
        __syncthreads();
        if (tid == 0) G = groups[g];
        __syncthreads();
        if (tid < G.n_slots) gs[tid] = occ ? (float)occ[G.orb[tid]] : 1.f;
        for (int s = 0; s < G.n_slots; ++s) {
            ps[s][tid] = valid ? __ldg(psi4 + (long long)G.orb[s] * N4 + x4) : make_float4(0.f, 0.f, 0.f, 0.f);
            as[s][tid] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        if (valid) {
#pragma unroll 4
            for (int k = 0; k < G.n_items; ++k) {
                const int item = G.first_item + k;
                const int2 sl = __ldg(item_slot + item);
                const float4 f = __ldg(phi4 + (long long)(item - item0) * N4 + x4);
                const float4 pj = ps[sl.y][tid];
                const float gj = gs[sl.y];
                float4 ai = as[sl.x][tid];
                ai.x = fmaf(gj * pj.x, f.x, ai.x);
                ai.y = fmaf(gj * pj.y, f.y, ai.y);
                ai.z = fmaf(gj * pj.z, f.z, ai.z);
                ai.w = fmaf(gj * pj.w, f.w, ai.w);
                as[sl.x][tid] = ai;
                if (sl.x != sl.y) {
                    const float4 pi = ps[sl.x][tid];
                    const float gi = gs[sl.x];
                    float4 aj = as[sl.y][tid];
                    aj.x = fmaf(gi * pi.x, f.x, aj.x);
                    aj.y = fmaf(gi * pi.y, f.y, aj.y);
                    aj.z = fmaf(gi * pi.z, f.z, aj.z);
                    aj.w = fmaf(gi * pi.w, f.w, aj.w);
                    as[sl.y][tid] = aj;
                }
            }
            for (int s = 0; s < G.n_slots; ++s) {
                float4 *dst = acc4 + (long long)G.orb[s] * N4 + x4;
                float4 o = *dst;
                const float4 d = as[s][tid];
                o.x += d.x;
                o.y += d.y;
                o.z += d.z;
                o.w += d.w;
                *dst = o;
            }
        }
    }
}

// psi (fp64) -> psi32 and per-vector max |value|.
__global__ void prep_kernel(const double *__restrict__ src, float *__restrict__ dst, float *__restrict__ vmax,
                            int n_vec, long long N) {
    const int v = blockIdx.y;
    float m = 0.f;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < N; x += (long long)gridDim.x * blockDim.x) {
        const float f = (float)src[(long long)v * N + x];
        dst[(long long)v * N + x] = f;
        m = fmaxf(m, fabsf(f));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(reinterpret_cast<int *>(vmax + v), __float_as_int(m));
}

__global__ void finalize_kernel(const float *__restrict__ acc, double *__restrict__ vx, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        vx[e] = -(double)acc[e];
}

__global__ void energy_add_kernel(const double *__restrict__ partial, int n, double factor, double *e_x) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s += partial[b];
        *e_x += factor * s;
    }
}

// Failure-path self-test: wait on an mbarrier phase that nothing completes; the
// bounded wait gives up and the status word records KX_ERR_TIMEOUT.
__global__ void selftest_wait_kernel(long long max_cycles, int *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !ptx::mbar_wait_bounded(&bar, 0, max_cycles)) atomicExch(status, KX_ERR_TIMEOUT);
}

size_t stage_bytes_of(int np) { return (size_t)2 * 128 * np * 2; }

int pass_stages(int np, bool with_mid) {
    const size_t v = (size_t)4 * np * np;
    const size_t avail = kSmemBudget - v - (with_mid ? stage_bytes_of(np) : 0);
    return (int)std::max<size_t>(1, std::min<size_t>(kMaxStages, avail / stage_bytes_of(np)));
}

size_t pass_smem(int np, int stages, bool with_mid) {
    return (size_t)4 * np * np + (size_t)(stages + (with_mid ? 1 : 0)) * stage_bytes_of(np) + 1024;
}

template <int PASS>
int launch_pass(const kx_plan *p, PassArgs a, int axis, cudaStream_t s, int *grid_out) {
    a.nc = p->n[axis];
    a.np = p->np[axis];
    a.Vs = p->d_Vs[axis];
    a.n1 = p->n[0];
    a.n2 = p->n[1];
    a.n3 = p->n[2];
    a.N = (long long)p->N;
    a.status = p->d_status;
    a.timeout_cycles = 4000000000LL;  // ~2 s at the SM clock
    const bool with_mid = (PASS == P_X1) && !a.energy_only;
    a.stages = pass_stages(a.np, with_mid);
    const size_t smem = pass_smem(a.np, a.stages, with_mid);
    KX_CUDA_TRY(cudaFuncSetAttribute(tc_pass_kernel<PASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long n_tiles = (a.total_rows + 127) / 128;
    const int grid = (int)std::max(1LL, std::min<long long>(n_tiles, (long long)p->num_sms));
    if (grid_out) *grid_out = grid;
    if (int rc = prof_begin(const_cast<kx_plan *>(p), PK_X3F + PASS, s)) return rc;
    tc_pass_kernel<PASS><<<grid, kThreads, smem, s>>>(a);
    KX_LAUNCH_CHECK("tc_pass_kernel launch");
    return prof_end(const_cast<kx_plan *>(p), s);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct TcLayout {
    float *psi32, *acc, *T0, *T1, *orb_max, *mx;
    double *partial;
};

TcLayout carve(kx_plan *p, int n_vec, long chunk, bool with_acc) {
    TcLayout L{};
    uint8_t *b = reinterpret_cast<uint8_t *>(p->ws.ptr);
    size_t off = 0;
    auto take = [&](size_t bytes) { uint8_t *r = b + off; off += align256(bytes); return r; };
    L.psi32 = (float *)take(sizeof(float) * (size_t)n_vec * p->N);
    L.acc = with_acc ? (float *)take(sizeof(float) * (size_t)n_vec * p->N) : nullptr;
    L.T0 = (float *)take(sizeof(float) * (size_t)chunk * p->N);
    L.T1 = (float *)take(sizeof(float) * (size_t)chunk * p->N);
    L.orb_max = (float *)take(sizeof(float) * (size_t)n_vec);
    L.mx = (float *)take(sizeof(float) * 4 * (size_t)chunk);
    L.partial = (double *)take(sizeof(double) * 4096);
    return L;
}

float fmax_sqrt(const kx_plan *p) {
    // bound of |f(Lambda) (V1^T y)| / max|y| used for the mid-pass split scale
    return (float)(p->fmax * std::sqrt((double)p->n[0]) * 1.0001);
}

// The five passes over R items: X3F writes T0, X2F T0->T1, X1 T1->T0, X2I
// T0->T1, X3I T1->T0 (or xout in vector mode).  mx holds four rows of per-item
// maxima, mx_stride apart.
int run_passes(kx_plan *p, PassArgs a, long R, float *T0, float *T1, float *mx, long mx_stride, double *ex,
               double *partial, bool energy_only, double *xout, cudaStream_t s) {
    int rc;
    float *mx1 = mx, *mx2 = mx + mx_stride, *mx3 = mx + 2 * mx_stride, *mx4 = mx + 3 * mx_stride;
    a.rows_pp = (long long)p->n[0] * p->n[1];
    a.total_rows = R * a.rows_pp;
    a.out = T0;
    a.out_max = mx1;
    if ((rc = launch_pass<P_X3F>(p, a, 2, s, nullptr))) return rc;

    a.rows_pp = (long long)p->n[2] * p->n[0];
    a.total_rows = R * a.rows_pp;
    a.in = T0;
    a.in_max = mx1;
    a.out = T1;
    a.out_max = mx2;
    if ((rc = launch_pass<P_X2F>(p, a, 1, s, nullptr))) return rc;

    a.rows_pp = (long long)p->n[2] * p->n[1];
    a.total_rows = R * a.rows_pp;
    a.in = T1;
    a.in_max = mx2;
    a.out = T0;
    a.out_max = mx3;
    a.e_partial = ex ? partial : nullptr;
    a.energy_only = energy_only ? 1 : 0;
    int grid = 0;
    if ((rc = launch_pass<P_X1>(p, a, 0, s, &grid))) return rc;
    if (ex) {
        if ((rc = prof_begin(p, PK_FINAL, s))) return rc;
        energy_add_kernel<<<1, 32, 0, s>>>(partial, grid, -0.5 * p->dV, ex);
        KX_LAUNCH_CHECK("energy_add_kernel launch");
        if ((rc = prof_end(p, s))) return rc;
    }
    a.e_partial = nullptr;
    a.energy_only = 0;
    if (energy_only) return KX_OK;

    a.rows_pp = (long long)p->n[2] * p->n[0];
    a.total_rows = R * a.rows_pp;
    a.in = T0;
    a.in_max = mx3;
    a.out = T1;
    a.out_max = mx4;
    if ((rc = launch_pass<P_X2I>(p, a, 1, s, nullptr))) return rc;

    a.rows_pp = (long long)p->n[0] * p->n[1];
    a.total_rows = R * a.rows_pp;
    a.in = T1;
    a.in_max = mx4;
    a.out = T0;
    a.out_max = nullptr;
    a.xout = xout;
    return launch_pass<P_X3I>(p, a, 2, s, nullptr);
}

}  // namespace

long tc_default_chunk(const kx_plan *p, int n_orb) {
    (void)n_orb;
    if (p->tune.chunk_pairs > 0) return p->tune.chunk_pairs;
    const size_t budget = (size_t)4 << 30;  // both chunk buffers together
    long c = (long)std::max<size_t>(1, budget / (2 * p->N * sizeof(float)));
    return std::max(1L, std::min<long>(c, 2048));
}

size_t tc_workspace_bytes(const kx_plan *p, int n_vec, long chunk) {
    return align256(sizeof(float) * (size_t)n_vec * p->N) * 2 + align256(sizeof(float) * (size_t)chunk * p->N) * 2 +
           align256(sizeof(float) * n_vec) + align256(sizeof(float) * 4 * chunk) + align256(sizeof(double) * 4096) +
           4096;
}

int tc_vx(kx_plan *p, int n_orb, const double *psi, const double *occ, double *vx, double *ex, bool energy_only,
          cudaStream_t s, long pair_begin, long pair_end) {
    int rc = ensure_pairs(p, n_orb, s, pair_begin, pair_end);
    if (rc) return rc;
    const std::vector<int> &first = p->h_group_first;  // n_groups + 1 entries
    const int n_groups = (int)first.size() - 1;
    const long P = first.back();
    long cap = tc_default_chunk(p, n_orb);
    for (int g = 0; g < n_groups; ++g) cap = std::max<long>(cap, first[g + 1] - first[g]);  // a group never splits
    const long chunk = std::max(1L, std::min<long>(cap, std::max(P, 1L)));
    rc = ensure_workspace(p, tc_workspace_bytes(p, n_orb, chunk));
    if (rc) return rc;
    TcLayout L = carve(p, n_orb, chunk, !energy_only);
    const long long N = (long long)p->N;

    KX_CUDA_TRY(cudaMemsetAsync(L.orb_max, 0, sizeof(float) * n_orb, s));
    {
        dim3 g((unsigned)std::min<long long>((N + 255) / 256, 64), (unsigned)n_orb);
        if ((rc = prof_begin(p, PK_PREP, s))) return rc;
        prep_kernel<<<g, 256, 0, s>>>(psi, L.psi32, L.orb_max, n_orb, N);
        KX_LAUNCH_CHECK("prep_kernel launch");
        if ((rc = prof_end(p, s))) return rc;
    }
    if (!energy_only) KX_CUDA_TRY(cudaMemsetAsync(L.acc, 0, sizeof(float) * (size_t)n_orb * N, s));
    if (ex) KX_CUDA_TRY(cudaMemsetAsync(ex, 0, sizeof(double), s));
    const int2 *pairs = reinterpret_cast<const int2 *>(p->d_pairs);
    const float mid_bound = fmax_sqrt(p);

    int g0 = 0;
    while (g0 < n_groups) {
        int g1 = g0 + 1;
        while (g1 < n_groups && first[g1 + 1] - first[g0] <= chunk) ++g1;
        const long c0 = first[g0];
        const long R = first[g1] - c0;
        KX_CUDA_TRY(cudaMemsetAsync(L.mx, 0, sizeof(float) * 4 * chunk, s));
        PassArgs a{};
        a.pairs = pairs + c0;
        a.psi32 = L.psi32;
        a.orb_max = L.orb_max;
        a.occ = occ;
        a.f32 = p->d_f32;
        a.mid_bound = mid_bound;
        if ((rc = run_passes(p, a, R, L.T0, L.T1, L.mx, chunk, ex, L.partial, energy_only, nullptr, s))) return rc;
        if (!energy_only) {
            const unsigned blocks = (unsigned)((N / 4 + kAccThreads - 1) / kAccThreads);
            if ((rc = prof_begin(p, PK_ACC, s))) return rc;
            acc_kernel<<<blocks, kAccThreads, 0, s>>>(L.T0, reinterpret_cast<const Group *>(p->d_groups), g0, g1,
                                                     (int)c0, reinterpret_cast<const int2 *>(p->d_item_slot),
                                                     L.psi32, occ, L.acc, N);
            KX_LAUNCH_CHECK("acc_kernel launch");
            if ((rc = prof_end(p, s))) return rc;
        }
        g0 = g1;
    }
    if (!energy_only) {
        const long long n = (long long)n_orb * N;
        if ((rc = prof_begin(p, PK_FINAL, s))) return rc;
        finalize_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 8LL * p->num_sms), 256, 0, s>>>(L.acc, vx, n);
        KX_LAUNCH_CHECK("finalize_kernel launch");
        if ((rc = prof_end(p, s))) return rc;
    }
    return KX_OK;
}

int selftest_wait(kx_plan *p, long long max_cycles, cudaStream_t s) {
    selftest_wait_kernel<<<1, 32, 0, s>>>(max_cycles, p->d_status);
    KX_LAUNCH_CHECK("selftest_wait_kernel launch");
    return KX_OK;
}

int tc_apply_fL(kx_plan *p, int n_rhs, const double *b, double *x, cudaStream_t s) {
    const long chunk = std::min<long>(tc_default_chunk(p, 1), n_rhs);
    int rc = ensure_workspace(p, tc_workspace_bytes(p, (int)chunk, chunk));
    if (rc) return rc;
    TcLayout L = carve(p, (int)chunk, chunk, false);
    const long long N = (long long)p->N;
    const float mid_bound = fmax_sqrt(p);
    for (long c0 = 0; c0 < n_rhs; c0 += chunk) {
        const long R = std::min<long>(chunk, n_rhs - c0);
        KX_CUDA_TRY(cudaMemsetAsync(L.orb_max, 0, sizeof(float) * R, s));
        KX_CUDA_TRY(cudaMemsetAsync(L.mx, 0, sizeof(float) * 4 * chunk, s));
        dim3 g((unsigned)std::min<long long>((N + 255) / 256, 64), (unsigned)R);
        if ((rc = prof_begin(p, PK_PREP, s))) return rc;
        prep_kernel<<<g, 256, 0, s>>>(b + c0 * N, L.psi32, L.orb_max, (int)R, N);
        KX_LAUNCH_CHECK("prep_kernel launch");
        if ((rc = prof_end(p, s))) return rc;
        PassArgs a{};
        a.rhs_mode = 1;
        a.f32 = p->d_f32;
        a.mid_bound = mid_bound;
        a.src_max = L.orb_max;
        a.in = L.psi32;
        if ((rc = run_passes(p, a, R, L.T0, L.T1, L.mx, chunk, nullptr, nullptr, false, x + c0 * N, s))) return rc;
    }
    return KX_OK;
}

// ---------------------------------------------------------------------------
// f(L) B without device allocation (kx_apply_fL_noalloc).
//
// Callers that cannot allocate device memory at the point of the call (their
// device memory was reserved up front by a pool allocator, or they run inside
// a solver loop that must not pay the device-wide synchronisation of
// cudaMalloc / cudaFree) get this variant: its scratch is the file-scope
// array below, so the call itself allocates nothing.  The array is part of
// this module's image: every GPU that loads it holds kNoAllocBytes until the
// process exits.  All calls share it and it keeps the previous call's
// contents; the per-vector maxima that must start at zero are cleared at every
// call.  Calls whose GPU work overlaps (two streams, or two host threads on one
// device) race on the array.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocMaxElems = (size_t)5 << 19;  // n_rhs * N limit per call (2,621,440 grid values)
constexpr size_t kNoAllocMaxVec = 8192;               // >= kNoAllocMaxElems / 512 (smallest N with n % 8 == 0)
constexpr size_t kNoAllocBytes = 3 * kNoAllocMaxElems * sizeof(float) + 5 * kNoAllocMaxVec * sizeof(float);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
void *g_noalloc_ptr[kNoAllocMaxDevices] = {};  // device address of the array, per device

// Set-up, once per device with that device current: the host-side name of the
// array is only a stand-in, so the kernels get the address the runtime reports.
int noalloc_scratch(int dev, void **out) {
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return set_error(KX_ERR_UNSUPPORTED, "kx_apply_fL_noalloc: device index beyond 63");
    if (g_noalloc_ptr[dev] == nullptr) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "kx_apply_fL_noalloc: cudaGetSymbolAddress of the static scratch");
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return KX_OK;
}

}  // namespace

size_t noalloc_max_elems() { return kNoAllocMaxElems; }

int tc_apply_fL_noalloc(kx_plan *p, int n_rhs, const double *b, double *x, cudaStream_t s) {
    if (p->precision != KX_F16X3)
        return set_error(KX_ERR_UNSUPPORTED, "kx_apply_fL_noalloc: needs a KX_F16X3 plan");
    const long long N = (long long)p->N;
    if ((size_t)n_rhs * (size_t)N > kNoAllocMaxElems)
        return set_error(KX_ERR_ARG, "kx_apply_fL_noalloc: n_rhs * N = " + std::to_string((size_t)n_rhs * N) +
                                         " exceeds the static scratch limit of " +
                                         std::to_string(kNoAllocMaxElems) + " grid values; split the call");
    int dev = -1;
    KX_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != p->device) return set_error(KX_ERR_ARG, "kx_apply_fL_noalloc: call on the plan's device");
    void *base = nullptr;
    if (int rc = noalloc_scratch(dev, &base)) return rc;
    const size_t elems = (size_t)n_rhs * (size_t)N;
    float *b32 = reinterpret_cast<float *>(base);
    float *T0 = b32 + elems;
    float *T1 = T0 + elems;
    float *src_max = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(base) +
                                               3 * kNoAllocMaxElems * sizeof(float));
    float *mx = src_max + kNoAllocMaxVec;  // four per-item maxima rows of kNoAllocMaxVec
    KX_CUDA_TRY(cudaMemsetAsync(src_max, 0, 5 * kNoAllocMaxVec * sizeof(float), s));
    dim3 g((unsigned)std::min<long long>((N + 255) / 256, 64), (unsigned)n_rhs);
    prep_kernel<<<g, 256, 0, s>>>(b, b32, src_max, n_rhs, N);
    KX_LAUNCH_CHECK("prep_kernel launch");
    PassArgs a{};
    a.rhs_mode = 1;
    a.f32 = p->d_f32;
    a.mid_bound = fmax_sqrt(p);
    a.src_max = src_max;
    a.in = b32;
    return run_passes(p, a, n_rhs, T0, T1, mx, (long)kNoAllocMaxVec, nullptr, nullptr, false, x, s);
}

}  // namespace kx
