// Fully periodic grids through the discrete Fourier transform: the FFT variant
// that Sec. 3 and Fig. 1 set the Kronecker form against.  On a periodic axis
// the centred stencil is a circulant matrix, diagonalised by the DFT with
// eigenvalues lambda_a(k) = (w0 + 2 sum_p w_p cos(2 pi p k / n_a)) / h_a^2, so
//     f(L) b = IDFT( f(lambda1 + lambda2 + lambda3) . DFT(b) ),
// the same operator as the Kronecker form with Fourier eigenvectors.  Per item
// (a pair density or a right-hand side) three passes, float32 complex:
//   A  per x3 plane: form the source, 2D transform along x1 and x2 in shared memory
//   B  per line along x3: transform, scale by f (and sum f |Y|^2 for the energy
//      by Parseval), inverse transform
//   C  per x3 plane: inverse 2D transform, real part / N.
// The sources are real, so only the spectrum columns k1 <= n1 / 2 are kept (the
// rest are conjugates), which halves pass B and the x2 transforms, and two real
// rows share one complex transform along x1.
// Each batch of line transforms is a mixed-radix (4, 2, 3, 5) Stockham FFT whose
// stages are spread over the CTA's threads (lines x butterflies); lines of 80
// points instead take a four-step transform (16 x 5) held in registers.
#include "kx_internal.h"

#include <cmath>
#include <vector>

namespace kx {
namespace {

constexpr int kFftLine = 32;  // lines per CTA in pass B (40 KB of shared memory at n3 = 80: 5 CTAs per SM)
constexpr int kFftPlaneThreads = 512;  // passes A and C: two planes (2 x 104 KB at 80^2) and 32 warps per SM

struct FftAxis {
    int n, nr;
    int radix[8];
};

struct FftGeom {
    FftAxis ax[3];
    int n1, n2, n3;
    int h1;              // n1 / 2 + 1: the spectrum columns k1 kept (the sources are real)
    long long N, n12, nh;  // nh = h1 n2 spectrum points per x3 plane
    const float2 *tw;  // per axis 128 entries: exp(-2 pi i t / n_a), t < n_a
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// x / d for x < 2^14 and 2 <= d <= 128 as a multiply-high by m = 2^32 / d + 1
// (checked exhaustively over that range); d == 1 is passed as m == 0.
__device__ __forceinline__ unsigned fast_div(unsigned x, unsigned m) { return m ? __umulhi(x, m) : x; }
__device__ __forceinline__ unsigned div_magic(unsigned d) { return d > 1 ? 0xFFFFFFFFu / d + 1u : 0u; }

// u = DFT_R(v) with W the twiddle table of the line (exp(-2 pi i t / n)),
// nR = n / R; sg = -1 conjugates (inverse).  Radix 2 and 4 by additions and
// multiplications by +-i, radix 3 and 5 from the table.
template <int R>
__device__ __forceinline__ void dft_small(float2 *v, const float2 *W, int nR, float sg) {
    if (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = make_float2(a.x + b.x, a.y + b.y);
        v[1] = make_float2(a.x - b.x, a.y - b.y);
    } else if (R == 4) {
        // (-i sg) (x, y) = (sg y, -sg x)
        const float2 a = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
        const float2 b = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
        const float2 c = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
        const float2 t = make_float2(v[1].x - v[3].x, v[1].y - v[3].y);
        const float2 d = make_float2(sg * t.y, -sg * t.x);
        v[0] = make_float2(a.x + c.x, a.y + c.y);
        v[2] = make_float2(a.x - c.x, a.y - c.y);
        v[1] = make_float2(b.x + d.x, b.y + d.y);
        v[3] = make_float2(b.x - d.x, b.y - d.y);
    } else {
        float2 u[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            u[q] = v[0];
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = W[((q * r) % R) * nR];
                w.y *= sg;
                const float2 t = cmul(v[r], w);
                u[q].x += t.x;
                u[q].y += t.y;
            }
        }
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = u[q];
    }
}

// One Stockham stage of radix R over nl lines at once, spread over the CTA:
// line l's element k sits at a[l * lstride + k * st] (scratch b, same
// layout).  lines_fast picks the task order: consecutive threads take
// consecutive lines (element stride st > 1: neighbouring lines are adjacent)
// or consecutive butterflies of one line (st == 1).
template <int R>
__device__ __forceinline__ void fft_stage(const float2 *a, float2 *b, int n, int Ns, int nl, int lstride, int st,
                                          bool lines_fast, const float2 *W, float sg) {
    const int nR = n / R, tstep = n / (Ns * R);
    const unsigned m_fast = div_magic(lines_fast ? nl : nR), m_ns = div_magic(Ns);
    for (int task = threadIdx.x; task < nl * nR; task += blockDim.x) {
        int l, j;
        if (lines_fast) {
            j = (int)fast_div(task, m_fast);
            l = task - j * nl;
        } else {
            l = (int)fast_div(task, m_fast);
            j = task - l * nR;
        }
        const float2 *al = a + l * lstride;
        float2 *bl = b + l * lstride;
        const int jq = (int)fast_div(j, m_ns), jj = j - jq * Ns;
        float2 v[R];
        v[0] = al[j * st];
        const int tw0 = jj * tstep;  // < n / R
#pragma unroll
        for (int r = 1; r < R; ++r) {
            float2 w = W[tw0 * r];   // jj r tstep < n
            w.y *= sg;
            v[r] = cmul(al[(j + r * nR) * st], w);
        }
        dft_small<R>(v, W, nR, sg);
        const int base = jq * Ns * R + jj;
#pragma unroll
        for (int q = 0; q < R; ++q) bl[(base + q * Ns) * st] = v[q];
    }
}

// ---- lines of 80 points in registers: 80 = 16 x 5 (four-step)
//
// With x_p,q = x[p + 16 q] (p < 16, q < 5):
//   X[k5 + 5 k16] = sum_p W80^(p k5) W16^(p k16) sum_q x_p,q W5^(q k5),
// so phase 1 takes each p's five values through a 5-point DFT and the twiddle
// W80^(p k5) (into the scratch buffer at k5 16 + p) and phase 2 takes each
// k5's sixteen values through a 16-point DFT (4 x 4 with twiddles W16^(b k4))
// into X.  Tasks are ordered lines first, so that with the padded plane rows
// (or the 64-line columns of pass B) consecutive threads touch distinct banks.
// W5 and W16 are the constants cos, sin of 2 pi k / 5 and 2 pi k / 16; W80
// comes from the line's twiddle table.  sg = -1 conjugates (inverse).
__device__ __forceinline__ void dft4_reg(float2 &v0, float2 &v1, float2 &v2, float2 &v3, float sg) {
    const float2 a = make_float2(v0.x + v2.x, v0.y + v2.y);
    const float2 b = make_float2(v0.x - v2.x, v0.y - v2.y);
    const float2 c = make_float2(v1.x + v3.x, v1.y + v3.y);
    const float2 t = make_float2(v1.x - v3.x, v1.y - v3.y);
    const float2 d = make_float2(sg * t.y, -sg * t.x);  // -i sg t
    v0 = make_float2(a.x + c.x, a.y + c.y);
    v2 = make_float2(a.x - c.x, a.y - c.y);
    v1 = make_float2(b.x + d.x, b.y + d.y);
    v3 = make_float2(b.x - d.x, b.y - d.y);
}

__device__ __forceinline__ void dft5_reg(float2 *x, float sg) {
    constexpr float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;  // cos 2pi/5, cos 4pi/5
    constexpr float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;   // sin 2pi/5, sin 4pi/5
    const float2 t1 = make_float2(x[1].x + x[4].x, x[1].y + x[4].y);
    const float2 t2 = make_float2(x[2].x + x[3].x, x[2].y + x[3].y);
    const float2 t3 = make_float2(x[1].x - x[4].x, x[1].y - x[4].y);
    const float2 t4 = make_float2(x[2].x - x[3].x, x[2].y - x[3].y);
    const float2 a1 = make_float2(x[0].x + c1 * t1.x + c2 * t2.x, x[0].y + c1 * t1.y + c2 * t2.y);
    const float2 a2 = make_float2(x[0].x + c2 * t1.x + c1 * t2.x, x[0].y + c2 * t1.y + c1 * t2.y);
    const float2 b1 = make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
    const float2 b2 = make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
    const float2 m1 = make_float2(sg * b1.y, -sg * b1.x);  // -i sg b1
    const float2 m2 = make_float2(sg * b2.y, -sg * b2.x);
    x[0] = make_float2(x[0].x + t1.x + t2.x, x[0].y + t1.y + t2.y);
    x[1] = make_float2(a1.x + m1.x, a1.y + m1.y);
    x[4] = make_float2(a1.x - m1.x, a1.y - m1.y);
    x[2] = make_float2(a2.x + m2.x, a2.y + m2.y);
    x[3] = make_float2(a2.x - m2.x, a2.y - m2.y);
}

// x[0..16) in natural order -> X[0..16) in natural order
__device__ __forceinline__ void dft16_reg(float2 *x, float sg) {
    // cos and sin of 2 pi k / 16, k = 0 .. 9 (the twiddle exponents b k4 <= 9)
    constexpr float C[10] = {1.f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508978f, 0.f,
                             -0.38268343236508978f, -0.70710678118654752f, -0.92387953251128674f, -1.f,
                             -0.92387953251128674f};
    constexpr float S[10] = {0.f, 0.38268343236508978f, 0.70710678118654752f, 0.92387953251128674f, 1.f,
                             0.92387953251128674f, 0.70710678118654752f, 0.38268343236508978f, 0.f,
                             -0.38268343236508978f};
    // columns b: 4-point DFTs of x[b], x[4 + b], x[8 + b], x[12 + b] (index a), then W16^(b k4)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        dft4_reg(x[b], x[4 + b], x[8 + b], x[12 + b], sg);
#pragma unroll
        for (int k4 = 1; k4 < 4; ++k4) {
            if (b == 0) continue;
            const float wr = C[b * k4], wi = -sg * S[b * k4];
            const float2 v = x[4 * k4 + b];
            x[4 * k4 + b] = make_float2(v.x * wr - v.y * wi, v.x * wi + v.y * wr);
        }
    }
    // rows k4: 4-point DFTs over b; X[k4 + 4 kb] from row k4's output kb
    float2 y[16];
#pragma unroll
    for (int k4 = 0; k4 < 4; ++k4) {
        float2 v0 = x[4 * k4], v1 = x[4 * k4 + 1], v2 = x[4 * k4 + 2], v3 = x[4 * k4 + 3];
        dft4_reg(v0, v1, v2, v3, sg);
        y[k4] = v0;
        y[k4 + 4] = v1;
        y[k4 + 8] = v2;
        y[k4 + 12] = v3;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = y[k];
}

// 80-point transforms of nl lines (layout as in fft_stage), a -> b -> a; returns a.
__device__ float2 *fft80_lines(float2 *a, float2 *b, int nl, int lstride, int st, const float2 *W, bool inv) {
    const float sg = inv ? -1.f : 1.f;
    const unsigned m_nl = div_magic(nl);
    for (int task = threadIdx.x; task < nl * 16; task += blockDim.x) {  // phase 1: (line, p)
        const int p = (int)fast_div(task, m_nl), l = task - p * nl;
        const float2 *al = a + l * lstride;
        float2 x[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) x[q] = al[(p + 16 * q) * st];
        dft5_reg(x, sg);
        float2 *bl = b + l * lstride;
        bl[p * st] = x[0];
#pragma unroll
        for (int k5 = 1; k5 < 5; ++k5) {
            float2 w = W[p * k5];
            w.y *= sg;
            bl[(16 * k5 + p) * st] = cmul(x[k5], w);
        }
    }
    __syncthreads();
    for (int task = threadIdx.x; task < nl * 5; task += blockDim.x) {  // phase 2: (line, k5)
        const int k5 = (int)fast_div(task, m_nl), l = task - k5 * nl;
        const float2 *bl = b + l * lstride + 16 * k5 * st;
        float2 x[16];
#pragma unroll
        for (int p = 0; p < 16; ++p) x[p] = bl[p * st];
        dft16_reg(x, sg);
        float2 *al = a + l * lstride;
#pragma unroll
        for (int k16 = 0; k16 < 16; ++k16) al[(k5 + 5 * k16) * st] = x[k16];
    }
    __syncthreads();
    return a;
}

// Stockham FFT of nl lines (see fft_stage for the layout) by the whole CTA;
// the inverse uses conjugate twiddles and is unnormalised.  Returns the buffer
// that holds the result (a or b, by the number of stages).  Every thread of
// the CTA must call it; it ends with a barrier.
__device__ float2 *fft_lines(float2 *a, float2 *b, const FftAxis &ax, int nl, int lstride, int st, const float2 *W,
                             bool inv) {
    if (ax.n == 80) return fft80_lines(a, b, nl, lstride, st, W, inv);
    const float sg = inv ? -1.f : 1.f;
    const bool lines_fast = st != 1;
    int Ns = 1;
    for (int s = 0; s < ax.nr; ++s) {
        const int R = ax.radix[s];
        if (R == 4)
            fft_stage<4>(a, b, ax.n, Ns, nl, lstride, st, lines_fast, W, sg);
        else if (R == 2)
            fft_stage<2>(a, b, ax.n, Ns, nl, lstride, st, lines_fast, W, sg);
        else if (R == 3)
            fft_stage<3>(a, b, ax.n, Ns, nl, lstride, st, lines_fast, W, sg);
        else
            fft_stage<5>(a, b, ax.n, Ns, nl, lstride, st, lines_fast, W, sg);
        __syncthreads();
        float2 *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

__device__ __forceinline__ void load_twiddles(const float2 *__restrict__ tw, float2 *Ws) {
    for (int i = threadIdx.x; i < 3 * 128; i += blockDim.x) Ws[i] = tw[i];
}

// Pass A: x3 plane blockIdx.x of item blockIdx.y; source psi_i psi_j (pairs) or src32.
__global__ void __launch_bounds__(kFftPlaneThreads) fft_plane_fwd_kernel(const FftGeom G, const int2 *__restrict__ pairs,
                                                            const float *__restrict__ src32, int rhs,
                                                            float2 *__restrict__ C) {
    extern __shared__ float2 fsm[];
    __shared__ float2 Ws[3 * 128];
    const int ld = G.n1 + 1;  // padded rows
    float2 *A = fsm, *B = fsm + (size_t)G.n2 * ld;
    const int x3 = blockIdx.x;
    const long long item = blockIdx.y;
    const float *p0, *p1 = nullptr;
    if (rhs) {
        p0 = src32 + item * G.N + x3 * G.n12;
    } else {
        const int2 ij = pairs[item];
        p0 = src32 + (long long)ij.x * G.N + x3 * G.n12;
        p1 = src32 + (long long)ij.y * G.N + x3 * G.n12;
    }
    load_twiddles(G.tw, Ws);
    const unsigned m_n1 = div_magic(G.n1);  // plane index e < 2^14: multiply-high division by n1
    // four loads in flight per thread before their values are stored
    for (int e0 = threadIdx.x; e0 < G.n12; e0 += 4 * blockDim.x) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * blockDim.x;
            v[u] = e < G.n12 ? (p1 ? __ldg(p0 + e) * __ldg(p1 + e) : __ldg(p0 + e)) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e >= G.n12) break;
            const int x2 = (int)fast_div(e, m_n1), x1 = e - x2 * G.n1;
            // rows 2j and 2j + 1 as the real and imaginary parts of packed row j
            float *z = reinterpret_cast<float *>(A + (x2 >> 1) * ld + x1);
            z[x2 & 1] = v[u];
            if (x2 == G.n2 - 1 && (x2 & 1) == 0) z[1] = 0.f;  // an odd last row pairs with zeros
        }
    }
    __syncthreads();
    // rows along x1: one complex transform per two real rows, Z = DFT(a + i b),
    // then A(k) = (Z(k) + conj Z(-k)) / 2 and B(k) = (Z(k) - conj Z(-k)) / 2i for
    // the kept columns k1 < h1 into the other buffer's rows 2j and 2j + 1
    const int n2p = (G.n2 + 1) / 2;
    float2 *Z = fft_lines(A, B, G.ax[0], n2p, ld, 1, Ws, false);
    float2 *R1 = (Z == A) ? B : A;
    {
        const unsigned m_h1 = div_magic(G.h1);
        for (int e = threadIdx.x; e < n2p * G.h1; e += blockDim.x) {
            const int j = (int)fast_div(e, m_h1), k = e - j * G.h1;
            const float2 z = Z[j * ld + k], zc = Z[j * ld + (k == 0 ? 0 : G.n1 - k)];
            R1[2 * j * ld + k] = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y - zc.y));
            if (2 * j + 1 < G.n2) R1[(2 * j + 1) * ld + k] = make_float2(0.5f * (z.y + zc.y), -0.5f * (z.x - zc.x));
        }
    }
    __syncthreads();
    // columns along x2 for k1 < h1 only: the source is real, so its spectrum is
    // Hermitian and the columns k1 > n1 / 2 are conjugates of kept ones
    const float2 *R2 = fft_lines(R1, Z, G.ax[1], G.h1, 1, ld, Ws + 128, false);
    float2 *dst = C + item * G.N + x3 * G.nh;  // [k2][k1 < h1]
    const unsigned m_h1 = div_magic(G.h1);
    for (int e = threadIdx.x; e < G.nh; e += blockDim.x) {
        const int k2 = (int)fast_div(e, m_h1);
        dst[e] = R2[k2 * ld + e - k2 * G.h1];
    }
}

// Pass B: kFftLine lines along x3 (plane positions blockIdx.x * kFftLine + l) of
// item blockIdx.y: transform, f scaling, energy sum, inverse transform.
__global__ void __launch_bounds__(256) fft_axis3_kernel(const FftGeom G, float2 *__restrict__ C,
                                                        const float *__restrict__ ftab,
                                                        const int2 *__restrict__ pairs,
                                                        const double *__restrict__ occ, int rhs, int energy_only,
                                                        double *__restrict__ e_part) {
    extern __shared__ float2 fsm[];
    __shared__ float2 Ws[3 * 128];
    __shared__ double red[8];
    float2 *A = fsm, *B = fsm + (size_t)G.n3 * kFftLine;
    const int tid = threadIdx.x;
    const long long item = blockIdx.y;
    const long long p0 = (long long)blockIdx.x * kFftLine;
    float2 *col = C + item * G.N + p0;
    load_twiddles(G.tw, Ws);
    for (int e0 = tid; e0 < G.n3 * kFftLine; e0 += 4 * blockDim.x) {  // e = x3 * kFftLine + l, four in flight
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * blockDim.x;
            const int x3 = e / kFftLine, l = e % kFftLine;
            v[u] = (e < G.n3 * kFftLine && p0 + l < G.nh) ? col[x3 * G.nh + l] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < G.n3 * kFftLine) A[e] = v[u];
        }
    }
    __syncthreads();
    float2 *Rr = fft_lines(A, B, G.ax[2], kFftLine, 1, kFftLine, Ws + 256, false);
    float2 *Or = (Rr == A) ? B : A;
    // energy by Parseval over the half spectrum: the columns 0 < k1 < n1 / 2 stand
    // for themselves and their conjugates (weight 2), k1 = 0 and k1 = n1 / 2 once
    float ef = 0.f;  // at most n3 * kFftLine / blockDim = 16 terms per thread
    const unsigned m_h1 = div_magic(G.h1);
    for (int k = tid; k < G.n3 * kFftLine; k += blockDim.x) {
        const int k3 = k / kFftLine, l = k % kFftLine;
        const int p = (int)p0 + l;  // < nh < 2^14
        float f = 0.f, wk = 0.f;
        if (p < G.nh) {
            const int k2 = (int)fast_div(p, m_h1), k1 = p - k2 * G.h1;
            f = __ldg(ftab + k3 * G.n12 + (long long)k2 * G.n1 + k1);
            wk = (k1 == 0 || 2 * k1 == G.n1) ? 1.f : 2.f;
        }
        const float2 y = Rr[k];
        ef = fmaf(f * wk, y.x * y.x + y.y * y.y, ef);
        Rr[k] = make_float2(y.x * f, y.y * f);
    }
    double e = (double)ef;
    __syncthreads();
    if (!energy_only) {
        const float2 *R2 = fft_lines(Rr, Or, G.ax[2], kFftLine, 1, kFftLine, Ws + 256, true);
        for (int k = tid; k < G.n3 * kFftLine; k += blockDim.x) {
            const int x3 = k / kFftLine, l = k % kFftLine;
            if (p0 + l < G.nh) col[x3 * G.nh + l] = R2[k];
        }
    }
    if (e_part != nullptr) {
        double w = 0.0;
        if (!rhs) {
            const int2 ij = pairs[item];
            w = (ij.x == ij.y) ? 1.0 : 2.0;
            if (occ) w *= occ[ij.x] * occ[ij.y];
        }
        e *= w;
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if ((tid & 31) == 0) red[tid >> 5] = e;
        __syncthreads();
        if (tid == 0) {
            double sum = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) sum += red[k];
            e_part[item * gridDim.x + blockIdx.x] = sum;
        }
    }
}

// Pass C: inverse 2D transform of x3 plane blockIdx.x of item blockIdx.y; real part / N
// into out32 (fp32) or out64 (fp64, right-hand-side mode).
__global__ void __launch_bounds__(kFftPlaneThreads) fft_plane_inv_kernel(const FftGeom G, const float2 *__restrict__ C,
                                                            float *__restrict__ out32, double *__restrict__ out64) {
    extern __shared__ float2 fsm[];
    __shared__ float2 Ws[3 * 128];
    const int ld = G.n1 + 1;
    float2 *A = fsm, *B = fsm + (size_t)G.n2 * ld;
    const int x3 = blockIdx.x;
    const long long item = blockIdx.y;
    const float2 *src = C + item * G.N + x3 * G.nh;  // [k2][k1 < h1]
    load_twiddles(G.tw, Ws);
    const unsigned m_n1 = div_magic(G.n1);  // plane indices < 2^14: multiply-high division
    const unsigned m_h1 = div_magic(G.h1);
    for (int e0 = threadIdx.x; e0 < G.nh; e0 += 4 * blockDim.x) {  // four loads in flight per thread
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * blockDim.x;
            v[u] = e < G.nh ? src[e] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e >= G.nh) break;
            const int k2 = (int)fast_div(e, m_h1);
            A[k2 * ld + e - k2 * G.h1] = v[u];
        }
    }
    __syncthreads();
    float2 *R1 = fft_lines(A, B, G.ax[1], G.h1, 1, ld, Ws + 128, true);  // kept columns: along x2
    float2 *Zp = (R1 == A) ? B : A;
    // two rows per complex inverse along x1: packed row j holds Z(k) = A(k) + i B(k)
    // for every k1, A and B the spectra of rows 2j and 2j + 1, whose columns
    // k1 > n1 / 2 are the conjugates of kept ones (the inverse along x3 and x2 of a
    // Hermitian spectrum leaves every row Hermitian in k1); the inverse of Z is
    // then row 2j in its real part and row 2j + 1 in its imaginary part
    const int n2p = (G.n2 + 1) / 2;
    for (int e = threadIdx.x; e < n2p * G.n1; e += blockDim.x) {
        const int j = (int)fast_div(e, m_n1), k = e - j * G.n1;
        const bool kept = k < G.h1;
        const int ks = kept ? k : G.n1 - k;
        float2 a = R1[2 * j * ld + ks];
        float2 b = (2 * j + 1 < G.n2) ? R1[(2 * j + 1) * ld + ks] : make_float2(0.f, 0.f);
        if (!kept) {
            a.y = -a.y;
            b.y = -b.y;
        }
        Zp[j * ld + k] = make_float2(a.x - b.y, a.y + b.x);
    }
    __syncthreads();
    const float2 *R2 = fft_lines(Zp, R1, G.ax[0], n2p, ld, 1, Ws, true);  // packed rows: along x1
    const float inv_n = 1.f / (float)G.N;
    const long long base = item * G.N + x3 * G.n12;
    for (int e = threadIdx.x; e < G.n12; e += blockDim.x) {
        const int x2 = (int)fast_div(e, m_n1);
        const float2 z = R2[(x2 >> 1) * ld + e - x2 * G.n1];
        const float v = ((x2 & 1) ? z.y : z.x) * inv_n;
        if (out64)
            out64[base + e] = (double)v;
        else
            out32[base + e] = v;
    }
}

// ex += factor sum part[0..count): fixed strided partial sums and a fixed tree.
__global__ void __launch_bounds__(1024) fft_energy_reduce_kernel(const double *__restrict__ part, long long count,
                                                                 double factor, double *__restrict__ ex) {
    __shared__ double red[1024];
    double s = 0.0;
    for (long long i = threadIdx.x; i < count; i += 1024) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = 512; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *ex += factor * red[0];
}

bool factor_235(int n, FftAxis &ax) {
    ax.n = n;
    ax.nr = 0;
    int m = n;
    while (m % 4 == 0) {
        ax.radix[ax.nr++] = 4;
        m /= 4;
    }
    for (int r : {2, 3, 5})
        while (m % r == 0) {
            if (ax.nr == 8) return false;
            ax.radix[ax.nr++] = r;
            m /= r;
        }
    return m == 1;
}

FftGeom geom(const kx_plan *p) {
    FftGeom G{};
    for (int a = 0; a < 3; ++a) factor_235(p->n[a], G.ax[a]);
    G.n1 = p->n[0];
    G.n2 = p->n[1];
    G.n3 = p->n[2];
    G.N = (long long)p->N;
    G.n12 = (long long)p->n[0] * p->n[1];
    G.h1 = p->n[0] / 2 + 1;
    G.nh = (long long)G.h1 * p->n[1];
    G.tw = reinterpret_cast<const float2 *>(p->d_fft_tw);
    return G;
}

size_t plane_smem(const kx_plan *p) { return sizeof(float2) * 2 * (size_t)p->n[1] * (p->n[0] + 1); }
size_t line_smem(const kx_plan *p) { return sizeof(float2) * 2 * (size_t)p->n[2] * kFftLine; }

}  // namespace

bool fft_supported(const int *n, const int *bc) {
    FftAxis ax;
    for (int a = 0; a < 3; ++a)  // the twiddle tables hold 128 entries per axis
        if (bc[a] != KX_PERIODIC || n[a] > 128 || !factor_235(n[a], ax)) return false;
    return sizeof(float2) * 2 * (size_t)n[1] * (n[0] + 1) <= 200 * 1024;
}

int fft_setup(kx_plan *p) {
    // twiddles exp(-2 pi i t / n_a) and the f table in DFT order, from float64 host arithmetic
    std::vector<float> tw(3 * 128 * 2, 0.f);
    for (int a = 0; a < 3; ++a)
        for (int t = 0; t < p->n[a]; ++t) {
            const double ang = 2.0 * M_PI * t / p->n[a];
            tw[(a * 128 + t) * 2] = (float)std::cos(ang);
            tw[(a * 128 + t) * 2 + 1] = (float)-std::sin(ang);
        }
    const int m = p->fd_order / 2;
    std::vector<double> w(m + 1, 0.0);
    double fm = 1.0;
    for (int i = 2; i <= m; ++i) fm *= i;
    for (int q = 1; q <= m; ++q) {
        double fmq = 1.0, fpq = 1.0;
        for (int i = 2; i <= m - q; ++i) fmq *= i;
        for (int i = 2; i <= m + q; ++i) fpq *= i;
        w[q] = 2.0 * ((q % 2) ? 1.0 : -1.0) * fm * fm / (double(q) * q * fmq * fpq);
        w[0] -= 2.0 / (double(q) * q);
    }
    std::vector<double> lam[3];
    for (int a = 0; a < 3; ++a) {
        lam[a].resize(p->n[a]);
        for (int k = 0; k < p->n[a]; ++k) {
            double s = w[0];
            for (int q = 1; q <= m; ++q) s += 2.0 * w[q] * std::cos(2.0 * M_PI * q * k / p->n[a]);
            lam[a][k] = s / (p->h[a] * p->h[a]);
        }
    }
    std::vector<float> f(p->N);
    const double om2 = p->omega * p->omega;
    for (int k3 = 0; k3 < p->n[2]; ++k3)
        for (int k2 = 0; k2 < p->n[1]; ++k2)
            for (int k1 = 0; k1 < p->n[0]; ++k1) {
                const double mu = -(lam[0][k1] + lam[1][k2] + lam[2][k3]);
                double v;
                if (p->kind == KX_SCREENED)
                    v = (mu > 0.0) ? -4.0 * M_PI * std::expm1(-mu / (4.0 * om2)) / mu : M_PI / om2;
                else
                    v = 4.0 * M_PI / mu;
                f[((size_t)k3 * p->n[1] + k2) * p->n[0] + k1] = (float)v;
            }
    KX_CUDA_TRY(cudaMalloc(&p->d_fft_tw, sizeof(float) * tw.size()));
    KX_CUDA_TRY(cudaMalloc(&p->d_fft_f, sizeof(float) * p->N));
    KX_CUDA_TRY(cudaMemcpy(p->d_fft_tw, tw.data(), sizeof(float) * tw.size(), cudaMemcpyHostToDevice));
    KX_CUDA_TRY(cudaMemcpy(p->d_fft_f, f.data(), sizeof(float) * p->N, cudaMemcpyHostToDevice));
    return KX_OK;
}

size_t fft_partial_count(const kx_plan *p, long chunk) {
    const long long groups = ((long long)(p->n[0] / 2 + 1) * p->n[1] + kFftLine - 1) / kFftLine;
    return (size_t)std::max<long long>(4096, groups * chunk);
}

int fft_passes(kx_plan *p, long R, const int2 *pairs, const float *src32, int rhs, const double *occ, float2 *C,
               float *out32, double *out64, double *ex, double *partial, bool energy_only, cudaStream_t s) {
    const FftGeom G = geom(p);
    const size_t ps = plane_smem(p), ls = line_smem(p);
    KX_CUDA_TRY(cudaFuncSetAttribute(fft_plane_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps));
    KX_CUDA_TRY(cudaFuncSetAttribute(fft_plane_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps));
    KX_CUDA_TRY(cudaFuncSetAttribute(fft_axis3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ls));
    int rc;
    const dim3 gp((unsigned)p->n[2], (unsigned)R);
    if ((rc = prof_begin(p, PK_FFT, s))) return rc;
    fft_plane_fwd_kernel<<<gp, kFftPlaneThreads, ps, s>>>(G, pairs, src32, rhs, C);
    KX_LAUNCH_CHECK("fft_plane_fwd_kernel launch");
    const unsigned groups = (unsigned)((G.nh + kFftLine - 1) / kFftLine);  // pass B: half-spectrum positions
    double *e_part = (ex != nullptr && !rhs) ? partial : nullptr;
    fft_axis3_kernel<<<dim3(groups, (unsigned)R), 256, ls, s>>>(G, C, p->d_fft_f, pairs, occ, rhs,
                                                                    energy_only ? 1 : 0, e_part);
    KX_LAUNCH_CHECK("fft_axis3_kernel launch");
    if (e_part) {
        fft_energy_reduce_kernel<<<1, 1024, 0, s>>>(partial, (long long)groups * R, -0.5 * p->dV / (double)G.N, ex);
        KX_LAUNCH_CHECK("fft_energy_reduce_kernel launch");
    }
    if (!energy_only) {
        fft_plane_inv_kernel<<<gp, kFftPlaneThreads, ps, s>>>(G, C, out32, out64);
        KX_LAUNCH_CHECK("fft_plane_inv_kernel launch");
    }
    return prof_end(p, s);
}

}  // namespace kx
