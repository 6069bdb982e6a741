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
//   warps 0-7   epilogue (TMEM lane quadrant = warp % 4, one tile row per
//               thread; warps 0-3 and 4-7 take alternate column blocks)
//   warps 8-15  producers: global fp32 -> scale -> fp16 hi/lo -> shared stage
//   warp 16     TMEM allocation and MMA issue (one thread)
// with an S-deep ring of shared A stages and two TMEM accumulator slots, so
// loads, MMAs and stores of consecutive tiles overlap.
#include "kx_internal.h"
#include "kx_tc_ptx.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>

namespace kx {
namespace {

enum PassKind { P_X3F = 0, P_X2F = 1, P_X1 = 2, P_X2I = 3, P_X3I = 4 };

constexpr int kEpiWarps = 8;   // two per TMEM lane quadrant, alternate 16/32-column blocks
constexpr int kProdWarps = 8;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kProdThreads = 32 * kProdWarps;
constexpr int kProdGroups = 2;                            // producer groups work on alternate tiles
constexpr int kGroupThreads = kProdThreads / kProdGroups;  // 128: one thread per row for the K-major pass
constexpr int kMmaWarp = kEpiWarps + kProdWarps;
constexpr int kThreads = 32 * (kEpiWarps + kProdWarps + 1);
constexpr int kMaxStages = 4;
constexpr size_t kSmemBudget = 222 * 1024;

// Optional per-role cycle counters (compile with -DKX_ROLE_CLOCKS): each CTA
// writes kClk counters to PassArgs::clk[blockIdx.x * kClk + k].
constexpr int kClk = 12;
#ifdef KX_ROLE_CLOCKS
long long *g_clkbuf = nullptr;
#define KX_CLK_NOW() clock64()
#define KX_CLK_ADD(k, t0) (clk_acc[(k)] += clock64() - (t0))
#else
#define KX_CLK_NOW() 0LL
#define KX_CLK_ADD(k, t0) ((void)(t0))
#endif

// Shared-memory layout of the A operand (no swizzle, 8x8 fp16 core matrices of
// 128 contiguous bytes).  Core matrices sit kCoreStride = 144 bytes apart
// (128 + 16 of padding) so that a warp writing one 16-byte row into each of
// eight neighbouring core matrices hits eight different bank groups.
//   MN-major (8 rows contiguous in a core-matrix row):
//     (m, k) at (m/8)*144 + (k/8)*(16*144) + (k%8)*16 + (m%8)*2
//     descriptor: K-direction offset 16*144, M-direction offset 144
//   K-major (8 k contiguous in a core-matrix row), nkc = np/8:
//     (m, k) at (m/8)*(nkc*144) + (k/8)*144 + (m%8)*16 + (k%8)*2
//     descriptor: K-direction offset 144, M-direction offset nkc*144
constexpr int kCoreStride = 144;
__host__ __device__ constexpr size_t a_half_bytes(int np) { return (size_t)np * 16 * kCoreStride / 8; }

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
    long long *clk;        // role counters (only with KX_ROLE_CLOCKS)
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

// Per-tile source descriptors, computed once per tile by the producers: for
// the MN-major passes one per group of 8 rows (row (m, k) of the group reads
// p0 + k * kstride, 8 consecutive rows contiguous), for the K-major pass one per
// row (chunk kc reads p0 + 8 kc).  p0 == nullptr marks rows past the end.
struct SrcDesc {
    const float *p0[128];
    const float *p1[16];  // second orbital of the pair product (X3F pair mode)
    float scale[128];
};

template <int PASS>
__device__ __forceinline__ void make_desc(const PassArgs &a, long long tile, SrcDesc &d, int ptid) {
    const long long n12 = (long long)a.n1 * a.n2;
    const int nd = (PASS == P_X1) ? 128 : 16;
    if (ptid >= nd) return;
    const long long R0 = tile * 128 + (PASS == P_X1 ? ptid : 8 * ptid);  // < 2^31: 32-bit division below
    if (R0 >= a.total_rows) {
        d.p0[ptid] = nullptr;
        if (PASS == P_X3F) d.p1[ptid] = nullptr;
        d.scale[ptid] = 0.f;
        return;
    }
    const unsigned rpp = (unsigned)a.rows_pp;
    const long long item = (unsigned)R0 / rpp, local = (unsigned)R0 % rpp;
    d.scale[ptid] = ldexpf(1.f, scale_exp(item_in_max<PASS>(a, item)));
    if (PASS == P_X1) {
        d.p0[ptid] = a.in + item * a.N + local * a.n1;
    } else if (PASS == P_X3F) {
        if (a.rhs_mode) {
            d.p0[ptid] = a.in + item * a.N + local;
            d.p1[ptid] = nullptr;
        } else {
            const int2 ij = a.pairs[item];
            d.p0[ptid] = a.psi32 + (long long)ij.x * a.N + local;
            d.p1[ptid] = a.psi32 + (long long)ij.y * a.N + local;
        }
    } else if (PASS == P_X2F || PASS == P_X2I) {
        const long long k3 = (unsigned)local / (unsigned)a.n1, x1 = (unsigned)local % (unsigned)a.n1;  // rows (k3, x1)
        d.p0[ptid] = a.in + item * a.N + k3 * n12 + x1;
    } else {  // P_X3I: rows = positions
        d.p0[ptid] = a.in + item * a.N + local;
    }
}

template <int PASS, int U, bool TWO>
__device__ __forceinline__ void produce_tile_u(const PassArgs &a, const SrcDesc &d, uint8_t *Ahi, uint8_t *Alo,
                                               int ptid) {
    const int np = a.np;
    const int nkc = np >> 3;
    const int ntask = 16 * np;  // 128 rows x np columns / 8
    const unsigned magic = (65536u + (unsigned)nkc - 1u) / (unsigned)nkc;  // t / nkc == (t * magic) >> 16 for t < 2^11
    const long long kstride = (PASS == P_X3F || PASS == P_X3I) ? (long long)a.n1 * a.n2 : (long long)a.n1;
    for (int t0 = ptid; t0 < ntask; t0 += kGroupThreads * U) {
        float v[U][8];
        float u[TWO ? U : 1][8];
        // issue every load of the batch first (padding tasks read nothing)
#pragma unroll
        for (int r = 0; r < U; ++r) {
            const int t = t0 + r * kGroupThreads;
            const float *p0 = nullptr;
            const float *p1 = nullptr;
            bool ok = false;
            if (t < ntask) {
                if (PASS == P_X1) {
                    // lanes walk the 8-value chunks of one row, then the next row: contiguous reads
                    const int m = (int)(((unsigned)t * magic) >> 16), kc = t - m * nkc;
                    p0 = d.p0[m];
                    ok = p0 != nullptr && kc * 8 < a.nc;
                    if (ok) p0 += kc * 8;
                } else {
                    // lanes walk the 16 row groups at one k, then the next k: 16 x 32 contiguous bytes
                    const int g = t & 15, k = t >> 4;
                    p0 = d.p0[g];
                    ok = p0 != nullptr && k < a.nc;
                    if (ok) {
                        p0 += k * kstride;
                        if (TWO) p1 = d.p1[g] + k * kstride;
                    }
                }
            }
            if (ok) {
                ld8(p0, v[r]);
                if (TWO) ld8(p1, u[TWO ? r : 0]);
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c) v[r][c] = 0.f;
                if (TWO) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) u[TWO ? r : 0][c] = 0.f;
                }
            }
        }
        // then scale, split and store (offsets and scales re-derived from t)
#pragma unroll
        for (int r = 0; r < U; ++r) {
            const int t = t0 + r * kGroupThreads;
            if (t >= ntask) continue;
            int off;
            float sc;
            if (PASS == P_X1) {
                const int m = (int)(((unsigned)t * magic) >> 16), kc = t - m * nkc;
                off = (m >> 3) * (nkc * kCoreStride) + kc * kCoreStride + (m & 7) * 16;
                sc = d.scale[m];
            } else {
                const int g = t & 15, k = t >> 4;
                off = g * kCoreStride + (k >> 3) * (16 * kCoreStride) + (k & 7) * 16;
                sc = d.scale[g];
            }
            float w[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) w[c] = (TWO ? v[r][c] * u[TWO ? r : 0][c] : v[r][c]) * sc;
            uint4 hi4, lo4;
            split8(w, hi4, lo4);
            *reinterpret_cast<uint4 *>(Ahi + off) = hi4;
            *reinterpret_cast<uint4 *>(Alo + off) = lo4;
        }
    }
}

// Producer side: stage one 128-row tile of the A operand (scaled, split).
// Task t covers 8 consecutive values: MN-major row group g = t%16 at k = t/16;
// K-major row m = t/nkc, chunk kc = t%nkc.  Consecutive lanes therefore read
// consecutive global addresses.  All loads of a batch of U tasks (a whole tile for n <= 96 when U = 12) are
// issued before any is converted, so each thread keeps U*32 bytes in flight.
template <int PASS>
__device__ __forceinline__ void produce_tile(const PassArgs &a, const SrcDesc &d, uint8_t *Ahi, uint8_t *Alo,
                                             int ptid) {
    if (PASS == P_X3F) {
        if (a.rhs_mode)
            produce_tile_u<PASS, 6, false>(a, d, Ahi, Alo, ptid);
        else
            produce_tile_u<PASS, 4, true>(a, d, Ahi, Alo, ptid);
    } else {
        produce_tile_u<PASS, 8, false>(a, d, Ahi, Alo, ptid);
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
    const uint32_t a_lbo = a_kmajor ? (uint32_t)kCoreStride : (uint32_t)(16 * kCoreStride);
    const uint32_t a_sbo = a_kmajor ? (uint32_t)((np >> 3) * kCoreStride) : (uint32_t)kCoreStride;
    const uint32_t a_step = 2 * a_lbo;  // one k-step = two core matrices along K
    // V stored as 8x8 core matrices, row block of 8 x-rows = np*16 bytes.
    //   forward  (B[x][k] = V[x][k]): MN-major, K (=x) stride np*16, N (=k) stride 128
    //   inverse  (B[k][x] = V[x][k]): K-major,  K (=k) stride 128,   N (=x) stride np*16
    const uint32_t b_lbo = inverse ? 128u : (uint32_t)(np * 16);
    const uint32_t b_sbo = inverse ? (uint32_t)(np * 16) : 128u;
    const uint32_t b_step = inverse ? 256u : (uint32_t)(np * 32);
    const int nks = np >> 4;
    // descriptors built once; a k-step advances the start-address field (16-byte units)
    const uint64_t ah0 = ptx::sdesc(a_hi, a_lbo, a_sbo), al0 = ptx::sdesc(a_lo, a_lbo, a_sbo);
    const uint64_t bh0 = ptx::sdesc(v_hi, b_lbo, b_sbo), bl0 = ptx::sdesc(v_lo, b_lbo, b_sbo);
    const uint64_t a_inc = a_step >> 4, b_inc = b_step >> 4;
    {
        uint64_t ah = ah0, al = al0, bh = bh0, bl = bl0;
        ptx::mma_f16(tmem_a, ah, bl, idesc, 0u);
        ptx::mma_f16(tmem_a, al, bh, idesc, 1u);
        for (int ks = 1; ks < nks; ++ks) {
            ah += a_inc;
            al += a_inc;
            bh += b_inc;
            bl += b_inc;
            ptx::mma_f16(tmem_a, ah, bl, idesc, 1u);
            ptx::mma_f16(tmem_a, al, bh, idesc, 1u);
        }
    }
    {
        uint64_t ah = ah0, bh = bh0;
        for (int ks = 0; ks < nks; ++ks) {
            if (ks & 1)
                ptx::mma_f16(tmem_b, ah, bh, idesc, ks > 1 ? 1u : 0u);
            else
                ptx::mma_f16(tmem_a, ah, bh, idesc, 1u);
            ah += a_inc;
            bh += b_inc;
        }
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

// The threads of one producer group agree on `ok` and have finished their
// previous tile (a named barrier of the group, then a vote through shared memory).
__device__ __forceinline__ bool producers_agree(bool ok, int *flag, int gtid, int bar_id) {
    if (gtid == 0) *flag = 1;
    ptx::named_bar(bar_id, kGroupThreads);
    if (!ok) *flag = 0;
    ptx::named_bar(bar_id, kGroupThreads);
    const bool r = *flag != 0;
    ptx::named_bar(bar_id, kGroupThreads);
    return r;
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
    uint64_t drain;
};

// X1 epilogue, inverse half of tile j: wait for its inverse MMA, unscale and
// store the row (float4 per 4 columns), track the maximum, release the slot.
__device__ __forceinline__ bool x1_inverse_half(const PassArgs &a, Bars &bars, uint32_t tmem, int q, int hcol, int j,
                                                int np, bool two_acc, bool valid, long long item, long long local,
                                                float unscale2, volatile int *abort) {
    const int b = j & 1;
    if (!wait_bar_warp(&bars.tfull2[b], (uint32_t)((j >> 1) & 1), a, abort)) return false;
    ptx::tc_fence_after();
    const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * 2 * np);
    const uint32_t tb = ta + (uint32_t)np;
    float my_max = 0.f;
    float *orow = a.out + item * a.N + local * a.n1;
    for (int c = hcol; c < (np >> 4); c += 2) {
        float v[16], vb[16];
        ptx::tmem_ld16x2(ta + 16 * c, tb + 16 * c, v, vb);
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {  // store each 8-column half that lies inside the row
            if (!valid || 16 * c + 8 * h2 >= a.nc) continue;
            float wv[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                wv[k] = (two_acc ? v[8 * h2 + k] + vb[8 * h2 + k] : v[8 * h2 + k]) * unscale2;
                my_max = fmaxf(my_max, fabsf(wv[k]));
            }
            float4 *dst = reinterpret_cast<float4 *>(orow + 16 * c + 8 * h2);
            dst[0] = make_float4(wv[0], wv[1], wv[2], wv[3]);
            dst[1] = make_float4(wv[4], wv[5], wv[6], wv[7]);
        }
    }
    track_max(a.out_max, item, my_max, valid);
    ptx::tc_fence_before();
    ptx::mbar_arrive(&bars.tempty[b]);
    return true;
}

template <int PASS>
__global__ void __launch_bounds__(kThreads, 1) tc_pass_kernel(const PassArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int np = a.np;
    const int S = a.stages;
    const size_t half_bytes = a_half_bytes(np);
    const size_t stage_bytes = 2 * half_bytes;  // hi + lo
    uint8_t *Vhi = smem;
    uint8_t *Vlo = Vhi + np * np * 2;
    uint8_t *stage0 = Vlo + np * np * 2;
    __shared__ Bars bars;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    __shared__ double s_red[kEpiWarps];
    __shared__ SrcDesc sdesc[kProdGroups];
    __shared__ int s_vote[kProdGroups];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool with_inv = (PASS == P_X1) && !a.energy_only;
#ifdef KX_ROLE_CLOCKS
    long long clk_acc[kClk] = {0};
#endif
    const uint32_t tcols = (4 * np <= 256) ? 256u : 512u;
    if (warp == kMmaWarp) {
        ptx::tmem_alloc(&tmem_slot, tcols);
        ptx::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            ptx::mbar_init(&bars.full[s], kGroupThreads);
            ptx::mbar_init(&bars.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&bars.tfull[b], 1);
            ptx::mbar_init(&bars.tempty[b], kEpiThreads);
            ptx::mbar_init(&bars.tfull2[b], 1);
        }
        ptx::mbar_init(&bars.mid_full, kEpiThreads);
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
            const long long tm0 = KX_CLK_NOW();
            for (int it = 0; it <= n_my && ok; ++it) {
                if (it < n_my) {
                    const int s = it % S, b = it & 1;
                    long long tw = KX_CLK_NOW();
                    ok = wait_bar(&bars.full[s], (uint32_t)((it / S) & 1), a, &s_abort);
                    KX_CLK_ADD(5, tw);
                    tw = KX_CLK_NOW();
                    if (ok && it >= 2) ok = wait_bar(&bars.tempty[b], (uint32_t)(((it >> 1) - 1) & 1), a, &s_abort);
                    KX_CLK_ADD(6, tw);
                    if (!ok) break;
                    ptx::tc_fence_after();
                    const uint32_t sA = ptx::smem_u32(stage0 + s * stage_bytes);
                    const uint32_t da = tmem + (uint32_t)(b * 2 * np);
                    issue_split_mma(da, da + (uint32_t)np, sA, sA + (uint32_t)half_bytes, PASS == P_X1, sVhi,
                                    sVlo, inv, np);
                    if (!with_inv) ptx::mma_commit(&bars.empty[s]);  // X1 keeps the stage for its mid operand
                    ptx::mma_commit(&bars.tfull[b]);
                }
                if (with_inv && it >= 1) {
                    // inverse of tile j: its mid operand sits in tile j's own A stage
                    const int j = it - 1, b = j & 1, sj = j % S;
                    const long long tw = KX_CLK_NOW();
                    ok = wait_bar(&bars.mid_full, (uint32_t)(j & 1), a, &s_abort);
                    KX_CLK_ADD(7, tw);
                    if (!ok) break;
                    ptx::tc_fence_after();
                    const uint32_t sM = ptx::smem_u32(stage0 + sj * stage_bytes);
                    const uint32_t da = tmem + (uint32_t)(b * 2 * np);
                    issue_split_mma(da, da + (uint32_t)np, sM, sM + (uint32_t)half_bytes, true, sVhi, sVlo, true,
                                    np);
                    ptx::mma_commit(&bars.empty[sj]);
                    ptx::mma_commit(&bars.tfull2[b]);
                }
            }
            KX_CLK_ADD(4, tm0);
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
        const int grp = ptid / kGroupThreads, gtid = ptid % kGroupThreads;
        const long long tp0 = KX_CLK_NOW();
        for (int it = grp; it < n_my; it += kProdGroups) {  // groups take alternate tiles
            const int s = it % S;
            long long tw = KX_CLK_NOW();
            bool ok = it < S || wait_bar(&bars.empty[s], (uint32_t)(((it / S) - 1) & 1), a, &s_abort);
            KX_CLK_ADD(1, tw);
            tw = KX_CLK_NOW();
            ok = producers_agree(ok, &s_vote[grp], gtid, 2 + 2 * grp);
            if (!ok) break;
            make_desc<PASS>(a, blockIdx.x + (long long)it * gridDim.x, sdesc[grp], gtid);
            ptx::named_bar(3 + 2 * grp, kGroupThreads);
            KX_CLK_ADD(2, tw);
            tw = KX_CLK_NOW();
            uint8_t *Ahi = stage0 + s * stage_bytes;
            produce_tile<PASS>(a, sdesc[grp], Ahi, Ahi + half_bytes, gtid);
            ptx::fence_proxy_async_smem();
            ptx::mbar_arrive(&bars.full[s]);
            KX_CLK_ADD(3, tw);
        }
        KX_CLK_ADD(0, tp0);
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3, hcol = warp >> 2;  // lane quadrant, column half
        const int m = 32 * q + lane;  // TMEM lane == tile row of this thread
        const int nch = np >> 4;      // 16-column chunks
        double e_acc = 0.0;
        bool prev_valid = false;  // X1: the tile whose inverse half is still pending
        long long prev_item = 0, prev_local = 0;
        float prev_unscale2 = 0.f;
        bool aborted = false;
        const long long te0 = KX_CLK_NOW();
        const unsigned rpp = (unsigned)a.rows_pp;
        // the per-item scale of a row is fetched one tile ahead (its loads are
        // dependent L2 round trips that would otherwise follow the MMA wait)
        auto row_in_max = [&](int j) {
            const long long R = (blockIdx.x + (long long)j * gridDim.x) * 128 + m;
            return (R < a.total_rows) ? item_in_max<PASS>(a, (unsigned)R / rpp) : 0.f;
        };
        float in_mx_next = n_my > 0 ? row_in_max(0) : 0.f;
        for (int it = 0; it < n_my; ++it) {
            const int b = it & 1;
            // row information and the per-item scale do not depend on the MMA:
            // fetch them (and X1's first f chunk) before waiting for it
            const long long tile = blockIdx.x + (long long)it * gridDim.x;
            const long long R = tile * 128 + m;  // < 2^31
            const bool valid = R < a.total_rows;
            const long long item = valid ? (unsigned)R / rpp : 0;
            const long long local = valid ? (unsigned)R % rpp : 0;
            const float in_mx = in_mx_next;
            if (it + 1 < n_my) in_mx_next = row_in_max(it + 1);
            float fpre[16];
            if (PASS == P_X1) {
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    if (valid && 16 * hcol + 8 * h2 < a.nc) {
                        ld8(a.f32 + local * a.n1 + 16 * hcol + 8 * h2, fpre + 8 * h2);
                    } else {
#pragma unroll
                        for (int k = 0; k < 8; ++k) fpre[8 * h2 + k] = 0.f;
                    }
                }
            }
            long long tw = KX_CLK_NOW();
            if (!wait_bar_warp(&bars.tfull[b], (uint32_t)((it >> 1) & 1), a, &s_abort)) break;
            KX_CLK_ADD(9, tw);
            tw = KX_CLK_NOW();
            ptx::tc_fence_after();
            const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * 2 * np);
            const uint32_t tb = ta + (uint32_t)np;
            const float unscale = ldexpf(1.f, -(scale_exp(in_mx) + kVScaleExp));
            float my_max = 0.f;

            if (PASS == P_X1) {
                // forward half of tile it: energy, f scaling, mid operand into the tile's own A stage
                const int e_mid = scale_exp(a.mid_bound * in_mx);
                const float s_mid = ldexpf(1.f, e_mid);
                double w = 0.0;
                if (valid && a.e_partial != nullptr && !a.rhs_mode) {
                    int2 ij = a.pairs[item];
                    w = (ij.x == ij.y) ? 1.0 : 2.0;
                    if (a.occ) w *= a.occ[ij.x] * a.occ[ij.y];
                }
                uint8_t *midh = stage0 + (it % S) * stage_bytes;
                float e_row = 0.f;
                for (int c = hcol; c < nch; c += 2) {
                    float fk[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) fk[k] = fpre[k];
                    // prefetch the next chunk's f while this one is processed
                    // (nc is a multiple of 8: each 8-column half is either in or out)
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        if (valid && 16 * (c + 2) + 8 * h2 < a.nc) {
                            ld8(a.f32 + local * a.n1 + 16 * (c + 2) + 8 * h2, fpre + 8 * h2);
                        } else {
#pragma unroll
                            for (int k = 0; k < 8; ++k) fpre[8 * h2 + k] = 0.f;
                        }
                    }
                    float v[16], vb[16];
                    ptx::tmem_ld16x2(ta + 16 * c, tb + 16 * c, v, vb);
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const float y = (two_acc ? v[k] + vb[k] : v[k]) * unscale;
                        e_row = fmaf(fk[k] * y, y, e_row);
                        v[k] = fk[k] * y * s_mid;
                    }
                    if (with_inv) {
#pragma unroll
                        for (int h2 = 0; h2 < 2; ++h2) {
                            uint4 hi, lo;
                            split8(v + 8 * h2, hi, lo);
                            const int off = (m >> 3) * ((np >> 3) * kCoreStride) + (2 * c + h2) * kCoreStride + (m & 7) * 16;
                            *reinterpret_cast<uint4 *>(midh + off) = hi;
                            *reinterpret_cast<uint4 *>(midh + half_bytes + off) = lo;
                        }
                    }
                }
                e_acc += w * (double)e_row;
                if (with_inv) {
                    ptx::fence_proxy_async_smem();
                    ptx::tc_fence_before();
                    ptx::mbar_arrive(&bars.mid_full);
                    KX_CLK_ADD(10, tw);
                    tw = KX_CLK_NOW();
                    // inverse half of the previous tile (its MMA ran while this tile's forward half was processed)
                    if (it >= 1) {
                        if (!x1_inverse_half(a, bars, tmem, q, hcol, it - 1, np, two_acc, prev_valid, prev_item,
                                             prev_local, prev_unscale2, &s_abort))
                            break;
                    }
                    KX_CLK_ADD(11, tw);
                    prev_valid = valid;
                    prev_item = item;
                    prev_local = local;
                    prev_unscale2 = ldexpf(1.f, -(e_mid + kVScaleExp));
                    continue;  // tile it's TMEM slot is released by its inverse half
                }
            } else {
                // transposed write: one column per store, consecutive lanes = consecutive rows;
                // row base and column stride are computed once per tile
                // output (row r, column c) at base(r) + c * ostride: [k3 or x3][position] or [k3][k2 or x2][x1]
                const long long ostride = (PASS == P_X3F || PASS == P_X3I) ? n12 : (long long)a.n1;
                long long obase = 0;
                if (valid) {
                    if (PASS == P_X3F || PASS == P_X3I) {
                        obase = item * a.N + local;
                    } else {
                        const long long k3 = (unsigned)local / (unsigned)a.n1;
                        const long long x1 = (unsigned)local % (unsigned)a.n1;
                        obase = item * a.N + k3 * n12 + x1;
                    }
                }
                for (int cb = 32 * hcol; cb < np; cb += 64) {
                    float v[32], vb[32];
                    const long long tl = KX_CLK_NOW();
                    if (cb + 32 <= np) {
                        ptx::tmem_ld32x2(ta + cb, tb + cb, v, vb);
                    } else {
                        ptx::tmem_ld16x2(ta + cb, tb + cb, v, vb);
                    }
                    KX_CLK_ADD(11, tl);
                    if (!valid) continue;
                    const int w = min(32, a.nc - cb);
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        if (k >= w) break;
                        const float y = (two_acc ? v[k] + vb[k] : v[k]) * unscale;
                        const long long dst = obase + (long long)(cb + k) * ostride;
                        if (PASS == P_X3I && a.rhs_mode) {
                            a.xout[dst] = (double)y;
                        } else {
                            my_max = fmaxf(my_max, fabsf(y));
                            a.out[dst] = y;
                        }
                    }
                }
                track_max(a.out_max, item, my_max, valid);
            }
            ptx::tc_fence_before();
            ptx::mbar_arrive(&bars.tempty[b]);
            KX_CLK_ADD(10, tw);
        }
        KX_CLK_ADD(8, te0);
        if (PASS == P_X1 && with_inv && n_my >= 1 && !s_abort)
            aborted = !x1_inverse_half(a, bars, tmem, q, hcol, n_my - 1, np, two_acc, prev_valid, prev_item, prev_local,
                                       prev_unscale2, &s_abort);
        (void)aborted;
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
#ifdef KX_ROLE_CLOCKS
    if (a.clk != nullptr) {
        long long *o = a.clk + (long long)blockIdx.x * kClk;
        if (warp == kMmaWarp && lane == 0) { o[4] = clk_acc[4]; o[5] = clk_acc[5]; o[6] = clk_acc[6]; o[7] = clk_acc[7]; }
        if (tid == kEpiThreads) { o[0] = clk_acc[0]; o[1] = clk_acc[1]; o[2] = clk_acc[2]; o[3] = clk_acc[3]; }
        if (tid == 0) { o[8] = clk_acc[8]; o[9] = clk_acc[9]; o[10] = clk_acc[10]; o[11] = clk_acc[11]; }
    }
#endif
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, tcols);
    }
}

// ---------------------------------------------------------------------------
// Slab kernel: the three middle mode products of Eq. 19 for one k3 slice (an
// n1 x n2 plane of one item) without leaving the SM.  Per unit (item, k3):
//   M1  A1[x1][x2] (MN-major, from global) x V2      -> D1[x1][k2]
//   B   D1 -> A2[k2][x1] (MN-major, written by the thread owning row x1)
//   M2  A2 x V1                                      -> D2[k2][k1]
//   C   energy sum f Y^2; mid = f Y -> A3[k2][k1] (K-major, own row)
//   M3  A3 x V1^T                                    -> D3[k2][x1]
//   D   D3 -> A4[x1][k2] (MN-major, written by the thread owning row k2)
//   M4  A4 x V2^T                                    -> D4[x1][x2]
//   E   D4 -> global slice [x2][x1] (coalesced), per-item maximum
// Two units are in flight: unit j uses TMEM slot, A buffer and epilogue
// warpgroup j & 1, so the two groups run their stage chains independently and
// the single MMA thread serves whichever group is ready.  Split scales are
// powers of two from bounds: each orthogonal mode product grows max|.| by at
// most sqrt(n), the scaling by at most fmax.
// ---------------------------------------------------------------------------
struct SlabArgs {
    int n1, n2, n3, np1, np2;
    long long N;
    long long total_units;  // items * n3
    const float *in;
    float *out;
    const __half *V1s, *V2s;
    const float *in_max;    // per item
    float *out_max;         // per item (nullable)
    const float *f32;
    float fmax, sq1, sq2;   // fmax, sqrt(n1), sqrt(n2) (each with a small margin)
    double *e_partial;
    const int2 *pairs;
    const double *occ;
    int rhs_mode;
    int stage_in;           // the input plane is bulk-copied into shared memory before it is split
    int *status;
    long long timeout_cycles;
    long long *clk;         // role counters (only with KX_ROLE_CLOCKS)
};

constexpr int kSlabProdThreads = 96;
constexpr int kSlabU = 8;            // producer loads in flight per thread
// Warp roles: 16 epilogue warps (warp w reads TMEM lane quadrant w % 4, the
// TMEM access rule; column half (w / 4) % 2; group w / 8), then 3 producer
// warps, then the MMA warp.
constexpr int kSlabEpiWarps = 16;
constexpr int kSlabGroupThreads = 256;
constexpr int kSlabMmaWarp = kSlabEpiWarps + kSlabProdThreads / 32;
constexpr int kSlabThreads = 32 * (kSlabMmaWarp + 1);

struct SlabBars {
    uint64_t full[2], empty[2], tfull[2], ready[2], in_full, drain;
};

__device__ __forceinline__ bool slab_wait(uint64_t *bar, uint32_t parity, const SlabArgs &a, volatile int *abort) {
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

__device__ __forceinline__ void store_split8(uint8_t *hi_base, uint8_t *lo_base, int off, const float *w) {
    uint4 h, l;
    split8(w, h, l);
    *reinterpret_cast<uint4 *>(hi_base + off) = h;
    *reinterpret_cast<uint4 *>(lo_base + off) = l;
}

// Per-unit constants of the epilogue: item, slice, the four split exponents and
// the pair's energy weight.
struct SlabUnit {
    long long item, k3;
    int e1, e2, e3, e4;
    double w;
};

__device__ __forceinline__ SlabUnit slab_unit(const SlabArgs &a, long long u) {
    SlabUnit r;
    r.item = (unsigned)u / (unsigned)a.n3;
    r.k3 = (unsigned)u % (unsigned)a.n3;
    const float b1 = __ldg(a.in_max + r.item);
    const float b2 = b1 * a.sq2, b3 = a.fmax * a.sq1 * b2, b4 = a.sq1 * b3;
    r.e1 = scale_exp(b1);
    r.e2 = scale_exp(b2);
    r.e3 = scale_exp(b3);
    r.e4 = scale_exp(b4);
    r.w = 0.0;
    if (a.e_partial != nullptr && !a.rhs_mode) {
        const int2 ij = a.pairs[r.item];
        r.w = (ij.x == ij.y) ? 1.0 : 2.0;
        if (a.occ) r.w *= a.occ[ij.x] * a.occ[ij.y];
    }
    return r;
}

// Epilogue stage B or D for one warp: D row m (a TMEM lane) becomes K column m
// of the next MN-major operand; 8 consecutive D columns (M values) per 16-byte
// store.  Rows m >= nrow (padding) give zeros; rows m >= nprow are not written.
__device__ __forceinline__ void slab_transpose_stage(uint32_t ta, uint32_t tb, int m, int h, int nrow, int nprow,
                                                     int ncol, bool two, float us, uint8_t *Ahi, uint8_t *Alo) {
    const int off_r = (m >> 3) * (16 * kCoreStride) + (m & 7) * 16;
    for (int c = 16 * h; c < ncol; c += 32) {
        float v[16], vb[16];
        ptx::tmem_ld16x2(ta + c, tb + c, v, vb);
        if (m < nprow) {
#pragma unroll
            for (int g8 = 0; g8 < 2; ++g8) {
                float w[8];
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    w[k] = (m < nrow) ? (two ? v[8 * g8 + k] + vb[8 * g8 + k] : v[8 * g8 + k]) * us : 0.f;
                store_split8(Ahi, Alo, ((c >> 3) + g8) * kCoreStride + off_r, w);
            }
        }
    }
}

__global__ void __launch_bounds__(kSlabThreads, 1) tc_slab_kernel(const SlabArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int np1 = a.np1, np2 = a.np2, npm = max(np1, np2);
    const size_t half_bytes = a_half_bytes(npm);
    uint8_t *V1hi = smem;
    uint8_t *V1lo = V1hi + np1 * np1 * 2;
    uint8_t *V2hi = V1lo + np1 * np1 * 2;
    uint8_t *V2lo = V2hi + np2 * np2 * 2;
    uint8_t *buf0 = V2lo + np2 * np2 * 2;  // two A buffers (hi | lo), one per TMEM slot
    float *sin = reinterpret_cast<float *>(buf0 + 4 * half_bytes);  // input plane [x2][x1] (stage_in)
    __shared__ SlabBars bars;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    __shared__ double s_red[kSlabEpiWarps];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
#ifdef KX_ROLE_CLOCKS
    long long clk_acc[kClk] = {0};
    const long long clk_t0 = clock64();
#endif
    if (warp == kSlabMmaWarp) {
        ptx::tmem_alloc(&tmem_slot, 512);
        ptx::tmem_relinquish();
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&bars.full[b], kSlabProdThreads);
            ptx::mbar_init(&bars.empty[b], 1);
            ptx::mbar_init(&bars.tfull[b], 1);
            ptx::mbar_init(&bars.ready[b], kSlabGroupThreads);
        }
        ptx::mbar_init(&bars.in_full, 1);
        ptx::mbar_init(&bars.drain, 1);
        ptx::fence_mbar_init();
        s_abort = 0;
    }
    {
        const uint4 *s1 = reinterpret_cast<const uint4 *>(a.V1s);
        const uint4 *s2 = reinterpret_cast<const uint4 *>(a.V2s);
        uint4 *d1 = reinterpret_cast<uint4 *>(V1hi);
        uint4 *d2 = reinterpret_cast<uint4 *>(V2hi);
        const int c1 = (4 * np1 * np1) / 16, c2 = (4 * np2 * np2) / 16;
        for (int i = tid; i < c1; i += blockDim.x) d1[i] = __ldg(s1 + i);
        for (int i = tid; i < c2; i += blockDim.x) d2[i] = __ldg(s2 + i);
    }
    ptx::fence_proxy_async_smem();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int n_my = (int)((a.total_units - blockIdx.x + gridDim.x - 1) / gridDim.x);
    const long long n12 = (long long)a.n1 * a.n2;

    if (warp == kSlabMmaWarp) {
        // ---------------------------------------------------------------- MMA issue
        // Polls both slots and issues the next product of whichever is ready:
        // M1 of unit j needs its A1 (full) and the slot's previous unit through
        // stage E; M2..M4 need the group's previous stage (ready).
        if (lane == 0) {
            const uint32_t sV1h = ptx::smem_u32(V1hi), sV1l = ptx::smem_u32(V1lo);
            const uint32_t sV2h = ptx::smem_u32(V2hi), sV2l = ptx::smem_u32(V2lo);
            int jn[2] = {0, 1}, sn[2] = {0, 0};
            bool ok = true;
            long long last = clock64();
            while (ok && (jn[0] < n_my || jn[1] < n_my)) {
                bool progressed = false;
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const int j = jn[g], st = sn[g];
                    if (j >= n_my) continue;
                    bool go;
                    if (st == 0)
                        go = ptx::mbar_test_wait(&bars.full[g], (uint32_t)((j >> 1) & 1)) &&
                             (j < 2 || ptx::mbar_test_wait(&bars.ready[g], 1u));
                    else
                        go = ptx::mbar_test_wait(&bars.ready[g], (uint32_t)((st - 1) & 1));
                    if (!go) continue;
                    ptx::tc_fence_after();
                    const uint32_t sA = ptx::smem_u32(buf0 + g * 2 * half_bytes);
                    const uint32_t da = tmem + (uint32_t)(g * 2 * npm);
                    if (st == 0)  // M1: A1 (MN-major) x V2 forward
                        issue_split_mma(da, da + (uint32_t)npm, sA, sA + (uint32_t)half_bytes, false, sV2h, sV2l,
                                        false, np2);
                    else if (st == 1)  // M2: A2 (MN-major) x V1 forward
                        issue_split_mma(da, da + (uint32_t)npm, sA, sA + (uint32_t)half_bytes, false, sV1h, sV1l,
                                        false, np1);
                    else if (st == 2)  // M3: A3 (K-major) x V1^T
                        issue_split_mma(da, da + (uint32_t)npm, sA, sA + (uint32_t)half_bytes, true, sV1h, sV1l,
                                        true, np1);
                    else  // M4: A4 (MN-major) x V2^T
                        issue_split_mma(da, da + (uint32_t)npm, sA, sA + (uint32_t)half_bytes, false, sV2h, sV2l,
                                        true, np2);
                    ptx::mma_commit(&bars.tfull[g]);
                    if (st == 3) ptx::mma_commit(&bars.empty[g]);
                    if (++sn[g] == 4) {
                        sn[g] = 0;
                        jn[g] += 2;
                    }
                    progressed = true;
                }
                const long long now = clock64();
                if (progressed) {
                    last = now;
                } else if (s_abort) {
                    ok = false;
                } else if (now - last > a.timeout_cycles) {
                    s_abort = 1;
                    atomicExch(a.status, KX_ERR_TIMEOUT);
                    ok = false;
                }
            }
#ifdef KX_ROLE_CLOCKS
            clk_acc[5] = 0;
#endif
            if (!ok) {
                ptx::mma_commit(&bars.drain);
                ptx::mbar_wait_bounded(&bars.drain, 0, a.timeout_cycles);
            }
        }
        __syncwarp();
    } else if (warp >= kSlabEpiWarps) {
        // ---------------------------------------------------------------- producers: A1 from global
        const int ptid = tid - kSlabEpiWarps * 32;
        const int ntask = 16 * np2;  // 16 row groups (x1) x np2 columns (x2)
        const int nlines = (int)((n12 * 4) >> 7);  // 128-byte lines of a slice (n1 % 8 == 0)
        const uint32_t plane_bytes = (uint32_t)(n12 * 4);
        auto plane = [&](int it) {
            const long long u = blockIdx.x + (long long)it * gridDim.x;
            const long long item = (unsigned)u / (unsigned)a.n3, k3 = (unsigned)u % (unsigned)a.n3;
            return a.in + item * a.N + k3 * n12;
        };
        // stage_in: one thread copies the plane of the next unit into shared memory
        // (pieces of at most 16 KB) as soon as the previous plane has been split
        auto issue_plane = [&](int it) {
            ptx::fence_proxy_async_smem();
            ptx::mbar_arrive_expect_tx(&bars.in_full, plane_bytes);
            const char *src = reinterpret_cast<const char *>(plane(it));
            char *dst = reinterpret_cast<char *>(sin);
            for (uint32_t o = 0; o < plane_bytes; o += 16384u)
                ptx::bulk_load(dst + o, src + o, min(16384u, plane_bytes - o), &bars.in_full);
        };
        int inflight = -1;  // unit whose plane copy thread 0 issued and has not yet waited for
        if (a.stage_in && ptid == 0 && n_my > 0) {
            issue_plane(0);
            inflight = 0;
        }
        for (int it = 0; it < n_my; ++it) {
            const int sl = it & 1;
            if (it + 2 < n_my) {
                // pull the plane of unit it+2 into L2 while this unit waits for its buffer
                const char *src = reinterpret_cast<const char *>(plane(it + 2));
                for (int l = ptid; l < nlines; l += kSlabProdThreads) ptx::prefetch_l2(src + ((long long)l << 7));
            }
            long long tw = KX_CLK_NOW();
            bool ok = it < 2 || slab_wait(&bars.empty[sl], (uint32_t)(((it >> 1) - 1) & 1), a, &s_abort);
            KX_CLK_ADD(1, tw);
            tw = KX_CLK_NOW();
            if (ok && a.stage_in) ok = slab_wait(&bars.in_full, (uint32_t)(it & 1), a, &s_abort);
            if (ok && ptid == 0) inflight = -1;
            ok = ok && !s_abort;
            // with stage_in the producers meet at a named barrier below, so they leave together
            if (a.stage_in) ok = ptx::named_bar_and(2, kSlabProdThreads, ok);
            if (!ok) break;
            const long long u = blockIdx.x + (long long)it * gridDim.x;
            const long long item = (unsigned)u / (unsigned)a.n3;
            const float sc = ldexpf(1.f, scale_exp(a.in_max[item]));
            uint8_t *Ahi = buf0 + sl * 2 * half_bytes;
            uint8_t *Alo = Ahi + half_bytes;
            if (a.stage_in) {
#pragma unroll 4
                for (int t = ptid; t < ntask; t += kSlabProdThreads) {
                    const int g = t & 15, k = t >> 4;
                    float v[8];
                    if (8 * g < a.n1 && k < a.n2) {
                        const float4 *src = reinterpret_cast<const float4 *>(sin + k * a.n1 + 8 * g);
                        const float4 x0 = src[0], x1 = src[1];
                        v[0] = x0.x * sc; v[1] = x0.y * sc; v[2] = x0.z * sc; v[3] = x0.w * sc;
                        v[4] = x1.x * sc; v[5] = x1.y * sc; v[6] = x1.z * sc; v[7] = x1.w * sc;
                    } else {
#pragma unroll
                        for (int c = 0; c < 8; ++c) v[c] = 0.f;
                    }
                    store_split8(Ahi, Alo, g * kCoreStride + (k >> 3) * (16 * kCoreStride) + (k & 7) * 16, v);
                }
                ptx::fence_proxy_async_smem();
                ptx::mbar_arrive(&bars.full[sl]);
                // every producer has finished reading the plane: it may be overwritten
                ptx::named_bar(2, kSlabProdThreads);
                if (ptid == 0 && it + 1 < n_my) {
                    issue_plane(it + 1);
                    inflight = it + 1;
                }
            } else {
                const float *slice = plane(it);
                for (int t0 = ptid; t0 < ntask; t0 += kSlabProdThreads * kSlabU) {
                    float v[kSlabU][8];
#pragma unroll
                    for (int r = 0; r < kSlabU; ++r) {
                        const int t = t0 + r * kSlabProdThreads;
                        const int g = t & 15, k = t >> 4;
                        if (t < ntask && 8 * g < a.n1 && k < a.n2) {
                            ld8(slice + (long long)k * a.n1 + 8 * g, v[r]);
                        } else {
#pragma unroll
                            for (int c = 0; c < 8; ++c) v[r][c] = 0.f;
                        }
                    }
#pragma unroll
                    for (int r = 0; r < kSlabU; ++r) {
                        const int t = t0 + r * kSlabProdThreads;
                        if (t >= ntask) continue;
                        const int g = t & 15, k = t >> 4;
#pragma unroll
                        for (int c = 0; c < 8; ++c) v[r][c] *= sc;
                        store_split8(Ahi, Alo, g * kCoreStride + (k >> 3) * (16 * kCoreStride) + (k & 7) * 16, v[r]);
                    }
                }
                ptx::fence_proxy_async_smem();
                ptx::mbar_arrive(&bars.full[sl]);
            }
            KX_CLK_ADD(2, tw);
        }
        // a plane copy still in flight after an early exit must land before the CTA leaves
        if (inflight >= 0) ptx::mbar_wait_bounded(&bars.in_full, (uint32_t)(inflight & 1), a.timeout_cycles);
    } else {
        // ---------------------------------------------------------------- epilogue: group g = warp / 8
        // Warp w of a group reads TMEM lanes 32*(w%4).. (its D rows) and the
        // 16-column chunks c = 16*h + 32*i, h = (w/4)%2.  tcgen05.ld is
        // warp-collective: every lane loads, only the stores are predicated per row.
        const int g = warp >> 3, q = warp & 3, h = (warp >> 2) & 1;
        const int m = 32 * q + lane;  // TMEM lane == D row
        const bool two1 = (np1 >> 4) > 1, two2 = (np2 >> 4) > 1;
        const int nkc1 = np1 >> 3;
        const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(g * 2 * npm);
        const uint32_t tb = ta + (uint32_t)npm;
        uint8_t *Ahi = buf0 + g * 2 * half_bytes;
        uint8_t *Alo = Ahi + half_bytes;
        double e_acc = 0.0;
        bool ok = true;
        for (int j = g; j < n_my && ok; j += 2) {
            long long tw = KX_CLK_NOW();
            const SlabUnit U = slab_unit(a, blockIdx.x + (long long)j * gridDim.x);
            KX_CLK_ADD(0, tw);
            // ---- B: D1[x1][k2] -> A2[k2][x1]
            tw = KX_CLK_NOW();
            ok = __all_sync(0xffffffffu, slab_wait(&bars.tfull[g], 0u, a, &s_abort));
            KX_CLK_ADD(9, tw);
            if (!ok) break;
            tw = KX_CLK_NOW();
            ptx::tc_fence_after();
            if (32 * q < np1)
                slab_transpose_stage(ta, tb, m, h, a.n1, np1, np2, two2, ldexpf(1.f, U.e2 - U.e1 - kVScaleExp), Ahi,
                                     Alo);
            ptx::fence_proxy_async_smem();
            ptx::tc_fence_before();
            ptx::mbar_arrive(&bars.ready[g]);
            KX_CLK_ADD(10, tw);
            // ---- C: D2[k2][k1] = Y: energy sum f Y^2, mid = f Y -> A3[k2][k1] (K-major, own row)
            {
                const bool rowC = m < a.n2;
                const float *frow = a.f32 + (U.k3 * a.n2 + m) * (long long)a.n1;
                // f(Lambda) of this warp's first chunk; each further chunk's is fetched
                // while the previous one is processed
                float fr[2][16];
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int c0 = 16 * h + 8 * hh;
                    if (rowC && c0 < a.n1) {
                        ld8(frow + c0, fr[0] + 8 * hh);
                    } else {
#pragma unroll
                        for (int k = 0; k < 8; ++k) fr[0][8 * hh + k] = 0.f;
                    }
                }
                tw = KX_CLK_NOW();
                ok = __all_sync(0xffffffffu, slab_wait(&bars.tfull[g], 1u, a, &s_abort));
                KX_CLK_ADD(9, tw);
                if (!ok) break;
                tw = KX_CLK_NOW();
                ptx::tc_fence_after();
                const float u2 = ldexpf(1.f, -(U.e2 + kVScaleExp));
                const float s3 = ldexpf(1.f, U.e3);
                const int off_r = (m >> 3) * (nkc1 * kCoreStride) + (m & 7) * 16;
                float e_row = 0.f;
#pragma unroll
                for (int r = 0; r < kMaxN / 32; ++r) {
                    const int c = 16 * h + 32 * r;
                    if (c >= np1) break;
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const int c0 = c + 32 + 8 * hh;
                        if (rowC && c0 < a.n1) {
                            const float4 *src = reinterpret_cast<const float4 *>(frow + c0);
                            const float4 x0 = __ldg(src), x1 = __ldg(src + 1);
                            fr[(r + 1) & 1][8 * hh + 0] = x0.x;
                            fr[(r + 1) & 1][8 * hh + 1] = x0.y;
                            fr[(r + 1) & 1][8 * hh + 2] = x0.z;
                            fr[(r + 1) & 1][8 * hh + 3] = x0.w;
                            fr[(r + 1) & 1][8 * hh + 4] = x1.x;
                            fr[(r + 1) & 1][8 * hh + 5] = x1.y;
                            fr[(r + 1) & 1][8 * hh + 6] = x1.z;
                            fr[(r + 1) & 1][8 * hh + 7] = x1.w;
                        } else {
#pragma unroll
                            for (int k = 0; k < 8; ++k) fr[(r + 1) & 1][8 * hh + k] = 0.f;
                        }
                    }
                    float v[16], vb[16];
                    ptx::tmem_ld16x2(ta + c, tb + c, v, vb);
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const float y = rowC ? (two1 ? v[k] + vb[k] : v[k]) * u2 : 0.f;
                        e_row = fmaf(fr[r & 1][k] * y, y, e_row);
                        v[k] = fr[r & 1][k] * y * s3;
                    }
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh)
                        store_split8(Ahi, Alo, off_r + ((c >> 3) + hh) * kCoreStride, v + 8 * hh);
                }
                if (rowC) e_acc += U.w * (double)e_row;
                ptx::fence_proxy_async_smem();
                ptx::tc_fence_before();
                ptx::mbar_arrive(&bars.ready[g]);
                KX_CLK_ADD(11, tw);
            }
            // ---- D: D3[k2][x1] -> A4[x1][k2]
            tw = KX_CLK_NOW();
            ok = __all_sync(0xffffffffu, slab_wait(&bars.tfull[g], 0u, a, &s_abort));
            KX_CLK_ADD(9, tw);
            if (!ok) break;
            tw = KX_CLK_NOW();
            ptx::tc_fence_after();
            if (32 * q < np2)
                slab_transpose_stage(ta, tb, m, h, a.n2, np2, np1, two1, ldexpf(1.f, U.e4 - U.e3 - kVScaleExp), Ahi,
                                     Alo);
            ptx::fence_proxy_async_smem();
            ptx::tc_fence_before();
            ptx::mbar_arrive(&bars.ready[g]);
            KX_CLK_ADD(3, tw);
            // ---- E: D4[x1][x2] -> slice [x2][x1] of the output, coalesced over x1
            tw = KX_CLK_NOW();
            ok = __all_sync(0xffffffffu, slab_wait(&bars.tfull[g], 1u, a, &s_abort));
            KX_CLK_ADD(9, tw);
            if (!ok) break;
            tw = KX_CLK_NOW();
            ptx::tc_fence_after();
            {
                const float u4 = ldexpf(1.f, -(U.e4 + kVScaleExp));
                const bool valid = m < a.n1;
                float *orow = a.out + U.item * a.N + U.k3 * n12 + m;
                float my_max = 0.f;
                if (32 * q < a.n1) {
                    for (int c = 16 * h; c < np2; c += 32) {
                        float v[16], vb[16];
                        ptx::tmem_ld16x2(ta + c, tb + c, v, vb);
                        if (!valid) continue;
#pragma unroll
                        for (int k = 0; k < 16; ++k) {
                            if (c + k < a.n2) {
                                const float y = (two2 ? v[k] + vb[k] : v[k]) * u4;
                                my_max = fmaxf(my_max, fabsf(y));
                                orow[(long long)(c + k) * a.n1] = y;
                            }
                        }
                    }
                }
                track_max(a.out_max, U.item, my_max, valid);
            }
            ptx::tc_fence_before();
            ptx::mbar_arrive(&bars.ready[g]);
            KX_CLK_ADD(7, tw);
        }
        if (a.e_partial != nullptr) {
            double e = e_acc;
            for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
            if (lane == 0) s_red[warp] = e;
            ptx::named_bar(1, kSlabEpiWarps * 32);
            if (tid == 0) {
                double sum = 0.0;
                for (int w = 0; w < kSlabEpiWarps; ++w) sum += s_red[w];
                a.e_partial[blockIdx.x] = sum;
            }
        }
    }
#ifdef KX_ROLE_CLOCKS
    if (a.clk != nullptr) {
        long long *o = a.clk + (long long)blockIdx.x * kClk;
        const long long tot = clock64() - clk_t0;
        if (warp == kSlabMmaWarp && lane == 0) { o[4] = tot; }
        if (tid == kSlabEpiWarps * 32) { o[5] = tot; o[1] = clk_acc[1]; o[2] = clk_acc[2]; }
        if (tid == 0) { o[8] = tot; o[0] = clk_acc[0]; o[9] = clk_acc[9]; o[10] = clk_acc[10]; o[11] = clk_acc[11]; o[3] = clk_acc[3]; o[7] = clk_acc[7]; }
    }
#endif
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == kSlabMmaWarp) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 512);
    }
}

// Accumulation of one chunk, group by group: one thread per four grid points
// visits the group's items in order, adding g_j psi_j phi_ij to orbital i and
// g_i psi_i phi_ij to orbital j in shared-memory partial sums (one per orbital
// slot of the group, <= kGroupSlots), then adds the partial sums into the fp32
// accumulators.  All of a group's global loads (phi of every item, psi and the
// old accumulator of every slot) are issued before the first is used.  Every
// accumulator element is owned by one thread per launch and chunks run in a
// fixed order, so the result is deterministic.
constexpr int kAccThreads = 128;
constexpr int kGroupItems = kOrbBlock * kOrbBlock;

__global__ void __launch_bounds__(kAccThreads) acc_kernel(const float *__restrict__ phi, const Group *__restrict__ groups,
                                                         int g0, int g1, int item0, const int2 *__restrict__ item_slot,
                                                         const float *__restrict__ psi32, const double *__restrict__ occ,
                                                         float *__restrict__ acc, long long N) {
    __shared__ float4 ps[kGroupSlots][kAccThreads];
    __shared__ float4 as[kGroupSlots][kAccThreads];
    __shared__ Group G;
    __shared__ float gs[kGroupSlots];
    __shared__ int2 sl_s[kGroupItems];
    const int tid = threadIdx.x;
    const long long N4 = N >> 2;
    const long long x4 = (long long)blockIdx.x * kAccThreads + tid;
    const bool valid = x4 < N4;
    const float4 *phi4 = reinterpret_cast<const float4 *>(phi);
    const float4 *psi4 = reinterpret_cast<const float4 *>(psi32);
    float4 *acc4 = reinterpret_cast<float4 *>(acc);
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int g = g0; g < g1; ++g) {
        __syncthreads();
        if (tid == 0) G = groups[g];
        __syncthreads();
        const int ns = G.n_slots, ni = G.n_items, fi = G.first_item;
        if (tid < ns) gs[tid] = occ ? (float)occ[G.orb[tid]] : 1.f;
        if (tid < ni) sl_s[tid] = item_slot[fi + tid];
        float4 f[kGroupItems], o[kGroupSlots];
#pragma unroll
        for (int k = 0; k < kGroupItems; ++k)
            f[k] = (valid && k < ni) ? __ldg(phi4 + (long long)(fi + k - item0) * N4 + x4) : z;
#pragma unroll
        for (int s = 0; s < kGroupSlots; ++s) {
            if (s < ns) {
                const long long off = (long long)G.orb[s] * N4 + x4;
                ps[s][tid] = valid ? __ldg(psi4 + off) : z;
                o[s] = valid ? acc4[off] : z;
                as[s][tid] = z;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kGroupItems; ++k) {
            if (k >= ni) break;
            const int2 sl = sl_s[k];
            const float4 pj = ps[sl.y][tid];
            const float gj = gs[sl.y];
            float4 ai = as[sl.x][tid];
            ai.x = fmaf(gj * pj.x, f[k].x, ai.x);
            ai.y = fmaf(gj * pj.y, f[k].y, ai.y);
            ai.z = fmaf(gj * pj.z, f[k].z, ai.z);
            ai.w = fmaf(gj * pj.w, f[k].w, ai.w);
            as[sl.x][tid] = ai;
            if (sl.x != sl.y) {
                const float4 pi = ps[sl.x][tid];
                const float gi = gs[sl.x];
                float4 aj = as[sl.y][tid];
                aj.x = fmaf(gi * pi.x, f[k].x, aj.x);
                aj.y = fmaf(gi * pi.y, f[k].y, aj.y);
                aj.z = fmaf(gi * pi.z, f[k].z, aj.z);
                aj.w = fmaf(gi * pi.w, f[k].w, aj.w);
                as[sl.y][tid] = aj;
            }
        }
        if (valid) {
#pragma unroll
            for (int s = 0; s < kGroupSlots; ++s) {
                if (s < ns) {
                    const float4 d = as[s][tid];
                    acc4[(long long)G.orb[s] * N4 + x4] =
                        make_float4(o[s].x + d.x, o[s].y + d.y, o[s].z + d.z, o[s].w + d.w);
                }
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

// Vx psi = -acc over n values (n % 4 == 0; both pointers 16-byte aligned).
__global__ void finalize_kernel(const float *__restrict__ acc, double *__restrict__ vx, long long n) {
    const float4 *a4 = reinterpret_cast<const float4 *>(acc);
    double2 *v2 = reinterpret_cast<double2 *>(vx);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (n >> 2);
         e += (long long)gridDim.x * blockDim.x) {
        const float4 x = __ldg(a4 + e);
        v2[2 * e] = make_double2(-(double)x.x, -(double)x.y);
        v2[2 * e + 1] = make_double2(-(double)x.z, -(double)x.w);
    }
}

// The same for an output that is only 8-byte aligned.
__global__ void finalize_scalar_kernel(const float *__restrict__ acc, double *__restrict__ vx, long long n) {
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

size_t stage_bytes_of(int np) { return 2 * a_half_bytes(np); }
constexpr size_t kStagingBytes = 0;

int pass_stages(int np, bool with_mid) {
    const size_t v = (size_t)4 * np * np;
    const size_t avail = kSmemBudget - v - kStagingBytes - (with_mid ? stage_bytes_of(np) : 0);
    return (int)std::max<size_t>(1, std::min<size_t>(kMaxStages, avail / stage_bytes_of(np)));
}

size_t pass_smem(int np, int stages, bool with_mid) {
    return (size_t)4 * np * np + (size_t)(stages + (with_mid ? 1 : 0)) * stage_bytes_of(np) + kStagingBytes + 1024;
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
#ifdef KX_ROLE_CLOCKS
    if (!g_clkbuf) cudaMallocManaged(&g_clkbuf, sizeof(long long) * kClk * 4096 * 6);
    a.clk = g_clkbuf + (long long)PASS * kClk * 4096;
#endif
    a.stages = pass_stages(a.np, false);  // X1's mid operand reuses its tile's A stage
    if (p->tune.pass_stages > 0) a.stages = std::min(a.stages, p->tune.pass_stages);
    const size_t smem = pass_smem(a.np, a.stages, false);
    KX_CUDA_TRY(cudaFuncSetAttribute(tc_pass_kernel<PASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long n_tiles = (a.total_rows + 127) / 128;
    const int grid = (int)std::max(1LL, std::min<long long>(n_tiles, (long long)p->num_sms));
    if (grid_out) *grid_out = grid;
    if (int rc = prof_begin(const_cast<kx_plan *>(p), PK_X3F + PASS, s)) return rc;
    tc_pass_kernel<PASS><<<grid, kThreads, smem, s>>>(a);
    KX_LAUNCH_CHECK("tc_pass_kernel launch");
    return prof_end(const_cast<kx_plan *>(p), s);
}

size_t slab_smem(const kx_plan *p) {
    const int np1 = p->np[0], np2 = p->np[1], npm = std::max(np1, np2);
    return (size_t)4 * np1 * np1 + (size_t)4 * np2 * np2 + 4 * a_half_bytes(npm) + 1024;
}

// The slab kernel holds V1, V2 and two split A buffers in shared memory.
constexpr size_t kSlabSmemMax = 227 * 1024 - 1024;  // opt-in maximum less static shared memory
bool slab_fits(const kx_plan *p) { return slab_smem(p) <= kSlabSmemMax; }

bool use_slab(const kx_plan *p) {
    if (const char *e = std::getenv("KX_SLAB")) return std::atoi(e) != 0;  // tuning override
    return p->tune.fuse_slab != 0;
}

// Mode 2 forward, mode 1 forward, f(Lambda) scaling (+ energy), mode 1 inverse
// and mode 2 inverse of R items in one launch; `in` holds the mode-3 forward
// output, `out` receives the input of the mode-3 inverse (both natural layout).
int launch_slab(kx_plan *p, long R, const float *in, const float *in_max, float *out, float *out_max,
                double *e_partial, const int2 *pairs, const double *occ, int rhs_mode, cudaStream_t s,
                int *grid_out) {
    SlabArgs a{};
    a.n1 = p->n[0];
    a.n2 = p->n[1];
    a.n3 = p->n[2];
    a.np1 = p->np[0];
    a.np2 = p->np[1];
    a.N = (long long)p->N;
    a.total_units = (long long)R * a.n3;
    a.in = in;
    a.out = out;
    a.V1s = p->d_Vs[0];
    a.V2s = p->d_Vs[1];
    a.in_max = in_max;
    a.out_max = out_max;
    a.f32 = p->d_f32;
    a.fmax = (float)(p->fmax * 1.0001);
    a.sq1 = (float)(std::sqrt((double)a.n1) * 1.0001);
    a.sq2 = (float)(std::sqrt((double)a.n2) * 1.0001);
    a.e_partial = e_partial;
    a.pairs = pairs;
    a.occ = occ;
    a.rhs_mode = rhs_mode;
    a.status = p->d_status;
    a.timeout_cycles = 4000000000LL;  // ~2 s at the SM clock
#ifdef KX_ROLE_CLOCKS
    if (!g_clkbuf) cudaMallocManaged(&g_clkbuf, sizeof(long long) * kClk * 4096 * 6);
    a.clk = g_clkbuf + 5LL * kClk * 4096;
#endif
    size_t smem = slab_smem(p);
    const size_t plane = (size_t)a.n1 * a.n2 * 4;
    a.stage_in = (smem + plane <= kSlabSmemMax) ? 1 : 0;
    if (a.stage_in) smem += plane;
    // at least 120 KB so that one CTA (and one 512-column TMEM allocation) sits on each SM
    smem = std::max<size_t>(smem, 120 * 1024);
    KX_CUDA_TRY(cudaFuncSetAttribute(tc_slab_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (int)std::max(1LL, std::min<long long>(a.total_units, (long long)p->num_sms));
    if (grid_out) *grid_out = grid;
    if (int rc = prof_begin(p, PK_SLAB, s)) return rc;
    tc_slab_kernel<<<grid, kSlabThreads, smem, s>>>(a);
    KX_LAUNCH_CHECK("tc_slab_kernel launch");
    return prof_end(p, s);
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
    const bool fft = p->precision == KX_FFT32;  // T1 holds complex values, more energy partials
    L.T0 = (float *)take(sizeof(float) * (size_t)chunk * p->N);
    L.T1 = (float *)take(sizeof(float) * (fft ? 2 : 1) * (size_t)chunk * p->N);
    L.orb_max = (float *)take(sizeof(float) * (size_t)n_vec);
    L.mx = (float *)take(sizeof(float) * 4 * (size_t)chunk);
    L.partial = (double *)take(sizeof(double) * (fft ? fft_partial_count(p, chunk) : 4096));
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

    if (!energy_only && slab_fits(p) && use_slab(p)) {
        // X2F, X1 and X2I fused: T0 -> T1 without the intermediate round trips
        int grid = 0;
        if ((rc = launch_slab(p, R, T0, mx1, T1, mx4, ex ? partial : nullptr, a.pairs, a.occ, a.rhs_mode, s,
                              &grid)))
            return rc;
        if (ex) {
            if ((rc = prof_begin(p, PK_FINAL, s))) return rc;
            energy_add_kernel<<<1, 32, 0, s>>>(partial, grid, -0.5 * p->dV, ex);
            KX_LAUNCH_CHECK("energy_add_kernel launch");
            if ((rc = prof_end(p, s))) return rc;
        }
        a.e_partial = nullptr;
        a.energy_only = 0;
        a.rows_pp = (long long)p->n[0] * p->n[1];
        a.total_rows = R * a.rows_pp;
        a.in = T1;
        a.in_max = mx4;
        a.out = T0;
        a.out_max = nullptr;
        a.xout = xout;
        return launch_pass<P_X3I>(p, a, 2, s, nullptr);
    }

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
    if (const char *e = std::getenv("KX_CHUNK_PAIRS")) {  // tuning override (pairs per chunk)
        const long v = std::atol(e);
        if (v > 0) return v;
    }
    const size_t budget = (size_t)4 << 30;  // both chunk buffers together
    long c = (long)std::max<size_t>(1, budget / (2 * p->N * sizeof(float)));
    return std::max(1L, std::min<long>(c, 2048));
}

size_t tc_workspace_bytes(const kx_plan *p, int n_vec, long chunk) {
    const bool fft = p->precision == KX_FFT32;
    return align256(sizeof(float) * (size_t)n_vec * p->N) * 2 + align256(sizeof(float) * (size_t)chunk * p->N) +
           align256(sizeof(float) * (fft ? 2 : 1) * (size_t)chunk * p->N) + align256(sizeof(float) * n_vec) +
           align256(sizeof(float) * 4 * chunk) + align256(sizeof(double) * (fft ? fft_partial_count(p, chunk) : 4096)) +
           4096;
}

// Vx psi rows [o0, o1) = -acc, then the plan's final-rows hook (if set).
int finalize_rows(kx_plan *p, const float *acc, double *vx, int o0, int o1, cudaStream_t s) {
    if (o1 <= o0) return KX_OK;
    const long long n = (long long)(o1 - o0) * (long long)p->N;
    const size_t off = (size_t)o0 * p->N;
    if (int rc = prof_begin(p, PK_FINAL, s)) return rc;
    if ((reinterpret_cast<uintptr_t>(vx + off) & 15) == 0)
        finalize_kernel<<<(unsigned)std::min<long long>((n / 4 + 255) / 256, 8LL * p->num_sms), 256, 0, s>>>(
            acc + off, vx + off, n);
    else
        finalize_scalar_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 8LL * p->num_sms), 256, 0, s>>>(
            acc + off, vx + off, n);
    KX_LAUNCH_CHECK("finalize_kernel launch");
    if (int rc = prof_end(p, s)) return rc;
    if (p->final_hook.fn) p->final_hook.fn(p->final_hook.ctx, o0, o1, s);
    return KX_OK;
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
    // fp64 -> fp32 copies and maxima of orbitals [o0, o1)
    auto prep_range = [&](int o0, int o1) -> int {
        if (o1 <= o0) return KX_OK;
        dim3 g((unsigned)std::min<long long>((N + 255) / 256, 64), (unsigned)(o1 - o0));
        if (int r = prof_begin(p, PK_PREP, s)) return r;
        prep_kernel<<<g, 256, 0, s>>>(psi + (size_t)o0 * N, L.psi32 + (size_t)o0 * N, L.orb_max + o0, o1 - o0, N);
        KX_LAUNCH_CHECK("prep_kernel launch");
        return prof_end(p, s);
    };
    // orbitals arriving in pieces: each is waited for and converted before the
    // first chunk that needs it (the multipole correction needs all of them first)
    const InputPieces &pc = p->in_pieces;
    const bool pieces = !pc.end.empty() && !energy_only && !mp_tc_eligible(p, n_orb, psi);
    int prepped = 0;  // pieces converted so far
    auto need = [&](int o_need) -> int {
        while (prepped < (int)pc.end.size() && (prepped == 0 ? 0 : pc.end[prepped - 1]) < o_need) {
            KX_CUDA_TRY(cudaStreamWaitEvent(s, pc.ready[prepped], 0));
            if (int r = prep_range(prepped == 0 ? 0 : pc.end[prepped - 1], pc.end[prepped])) return r;
            ++prepped;
        }
        return KX_OK;
    };
    if (pieces) {
        if (!pc.end.empty() && pc.end.back() < n_orb) return set_error(KX_ERR_ARG, "input pieces do not cover the orbitals");
    } else {
        for (size_t k = 0; k < pc.ready.size(); ++k) KX_CUDA_TRY(cudaStreamWaitEvent(s, pc.ready[k], 0));
        if ((rc = prep_range(0, n_orb))) return rc;
    }
    auto piece_of = [&](int o) {
        int k = 0;
        while (k + 1 < (int)pc.end.size() && pc.end[k] <= o) ++k;
        return k;
    };
    const std::vector<int> &maxorb = p->h_group_maxorb;
    if (ex) KX_CUDA_TRY(cudaMemsetAsync(ex, 0, sizeof(double), s));
    if (!energy_only) {
        // with multipole boundary values the accumulator starts from the boundary
        // correction (tensor-core form), otherwise from zero
        if (mp_tc_eligible(p, n_orb, psi)) {
            if ((rc = mp_correct_into_acc(p, n_orb, psi, occ, L.acc, ex, s))) return rc;
        } else {
            KX_CUDA_TRY(cudaMemsetAsync(L.acc, 0, sizeof(float) * (size_t)n_orb * N, s));
        }
    }
    const int2 *pairs = reinterpret_cast<const int2 *>(p->d_pairs);
    const float mid_bound = fmax_sqrt(p);

    // pairs a chunk of a host-buffer call holds before it may end at a finished
    // row block (KX_ROW_CHUNK overrides: comparison runs)
    int row_chunk = 384;
    if (const char *e = std::getenv("KX_ROW_CHUNK")) row_chunk = std::max(1, std::atoi(e));
    // row_end[g]: groups [0, g) finish a row block (group g - 1 is the last one of
    // some orbital); tail: that row block is among the last three
    std::vector<char> row_end((size_t)n_groups + 1, 0), tail((size_t)n_groups + 1, 0);
    if (pieces)
        for (int o = 0; o < n_orb; ++o) {
            const int g = p->h_orb_last[o] + 1;
            if (g < 1 || g > n_groups) continue;
            row_end[g] = 1;
            if (o >= n_orb - 3 * kOrbBlock) tail[g] = 1;
        }
    int g0 = 0, o_fin = 0;
    while (g0 < n_groups) {
        int g1 = g0 + 1;
        while (g1 < n_groups && first[g1 + 1] - first[g0] <= chunk) {
            if (pieces) {
                // the first two pieces each end a chunk (their successors are still
                // copying); later pieces have arrived by the time they are needed.
                // A chunk ends where a row block becomes final once it holds
                // row_chunk pairs (at every one of the last three), so that
                // finished rows are copied back while the rest computes
                const int pg0 = piece_of(maxorb[g0]);
                if (pg0 < 2 && piece_of(maxorb[g1]) > pg0) break;
                if (row_end[g1] && (first[g1] - first[g0] >= row_chunk || tail[g1])) break;
            }
            ++g1;
        }
        if (pieces) {
            int o_need = 0;
            for (int g = g0; g < g1; ++g) o_need = std::max(o_need, maxorb[g] + 1);
            if ((rc = need(o_need))) return rc;
        }
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
        if (p->precision == KX_FFT32)
            rc = fft_passes(p, R, pairs + c0, L.psi32, 0, occ, reinterpret_cast<float2 *>(L.T1), L.T0, nullptr, ex,
                            L.partial, energy_only, s);
        else
            rc = run_passes(p, a, R, L.T0, L.T1, L.mx, chunk, ex, L.partial, energy_only, nullptr, s);
        if (rc) return rc;
        if (!energy_only) {
            const unsigned blocks = (unsigned)((N / 4 + kAccThreads - 1) / kAccThreads);
            if ((rc = prof_begin(p, PK_ACC, s))) return rc;
            acc_kernel<<<blocks, kAccThreads, 0, s>>>(L.T0, reinterpret_cast<const Group *>(p->d_groups), g0, g1,
                                                     (int)c0, reinterpret_cast<const int2 *>(p->d_item_slot),
                                                     L.psi32, occ, L.acc, N);
            KX_LAUNCH_CHECK("acc_kernel launch");
            if ((rc = prof_end(p, s))) return rc;
        }
        if (!energy_only) {
            // rows whose last group is done are final: negate them into vx now
            int o_done = o_fin;
            while (o_done < n_orb && p->h_orb_last[o_done] < g1) ++o_done;
            if ((rc = finalize_rows(p, L.acc, vx, o_fin, o_done, s))) return rc;
            o_fin = o_done;
        }
        g0 = g1;
    }
    if (pieces && (rc = need(n_orb))) return rc;  // every piece is on the device when the call's work ends
    if (!energy_only) return finalize_rows(p, L.acc, vx, o_fin, n_orb, s);
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
        if (p->precision == KX_FFT32)
            rc = fft_passes(p, R, nullptr, L.psi32, 1, nullptr, reinterpret_cast<float2 *>(L.T1), nullptr, x + c0 * N,
                            nullptr, nullptr, false, s);
        else
            rc = run_passes(p, a, R, L.T0, L.T1, L.mx, chunk, nullptr, nullptr, false, x + c0 * N, s);
        if (rc) return rc;
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

// The host-side name of the array is only a stand-in, so the kernels get the
// address the runtime reports for the current device.  It is looked up on
// every call (the lookup allocates nothing): a cached address would outlive a
// cudaDeviceReset, after which the module and its array are loaded anew.  On
// the first call on a device the lookup may load this module's device code,
// and the array with it, like any first launch from the module.
int noalloc_scratch(void **out) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "kx_apply_fL_noalloc: cudaGetSymbolAddress of the static scratch");
    *out = ptr;
    return KX_OK;
}

}  // namespace

size_t noalloc_max_elems() { return kNoAllocMaxElems; }

#ifdef KX_ROLE_CLOCKS
}  // namespace kx
// managed buffer written by the last launch of each pass (experiment builds only)
extern "C" long long *kx_debug_role_clocks() { return kx::g_clkbuf; }
namespace kx {
#endif

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
    if (int rc = noalloc_scratch(&base)) return rc;
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
