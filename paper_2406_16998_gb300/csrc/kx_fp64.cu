// Plain float64 Kronecker path on the CUDA cores: the accuracy reference on the
// GPU and the denominator of the tensor-core speed-up.
//
// For a chunk of R right-hand sides (pair products rho_ij = psi_i psi_j, or
// caller vectors), Sec. 3 Eq. 19 is applied as six mode products with Vk^T
// (forward) and Vk (inverse), with the Hadamard scaling by f(Lambda) between
// them.  Eq. 3-5 then accumulate (Vx psi)_i -= g_j psi_j phi_ij and
// (Vx psi)_j -= g_i psi_i phi_ij in a fixed pair order per grid point.
#include "kx_internal.h"

#include <algorithm>

namespace kx {
namespace {

constexpr int kTQ = 64;        // columns (pencils) per CTA
constexpr int kModeThreads = 256;

// out[o][c][i] = sum_k M[k][c] in[o][k][i]   with M = V (forward) or V^T (inverse),
// viewing each of the R grid vectors as [outer][n][inner] along `axis`.
// Pencils ("columns") are q = o*inner + i, kTQ of them per CTA.  Index work is
// kept off the per-element path: each thread finds the (o, i) of its one
// pencil with a single 32-bit division, then walks k with a fixed stride;
// the V copy and the contiguous (inner == 1) tiles use 2D loops.
__global__ void __launch_bounds__(kModeThreads) mode_f64_kernel(const double *__restrict__ in,
                                                               double *__restrict__ out, long long n_cols,
                                                               int n, long long inner,
                                                               const double *__restrict__ V, int inverse) {
    extern __shared__ double sm[];
    double *Ms = sm;                 // n*n: Ms[k*n + c]
    double *Ts = sm + n * n;         // n*(kTQ+1): Ts[k*(kTQ+1) + q]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int kWarps = kModeThreads / 32;
    for (int k = warp; k < n; k += kWarps)
        for (int c = lane; c < n; c += 32) Ms[k * n + c] = inverse ? V[c * n + k] : V[k * n + c];
    const int ld = kTQ + 1;
    const long long q0 = (long long)blockIdx.x * kTQ;
    const int nq = (int)min((long long)kTQ, n_cols - q0);
    const int ql = tid % kTQ, cg = tid / kTQ;  // this thread's pencil and column group (4 groups)
    // element (q, k) sits at o*n*inner + k*inner + i
    long long base = 0;
    if (inner == 1) {
        // pencils are contiguous rows of n values: warps take rows, lanes take k
        const double *src = in + q0 * n;
        for (int r = warp; r < nq; r += kWarps)
            for (int k = lane; k < n; k += 32) Ts[k * ld + r] = src[(long long)r * n + k];
    } else {
        if (ql < nq) {
            const unsigned q = (unsigned)(q0 + ql), in32 = (unsigned)inner;  // n_cols < 2^31
            const unsigned o = q / in32, i = q - o * in32;
            base = (long long)o * n * inner + i;
            for (int k = cg; k < n; k += kModeThreads / kTQ) Ts[k * ld + ql] = in[base + (long long)k * inner];
        }
    }
    __syncthreads();
    double acc[kMaxN / 4];
#pragma unroll
    for (int u = 0; u < kMaxN / 4; ++u) acc[u] = 0.0;
    if (ql < nq) {
        for (int k = 0; k < n; ++k) {
            double a = Ts[k * ld + ql];
#pragma unroll
            for (int u = 0; u < kMaxN / 4; ++u) {
                int c = cg + 4 * u;
                if (c < n) acc[u] = fma(Ms[k * n + c], a, acc[u]);
            }
        }
    }
    __syncthreads();
    if (ql < nq) {
#pragma unroll
        for (int u = 0; u < kMaxN / 4; ++u) {
            int c = cg + 4 * u;
            if (c < n) Ts[c * ld + ql] = acc[u];
        }
    }
    __syncthreads();
    if (inner == 1) {
        double *dst = out + q0 * n;
        for (int r = warp; r < nq; r += kWarps)
            for (int c = lane; c < n; c += 32) dst[(long long)r * n + c] = Ts[c * ld + r];
    } else if (ql < nq) {
        for (int c = cg; c < n; c += kModeThreads / kTQ) out[base + (long long)c * inner] = Ts[c * ld + ql];
    }
}

// B[r][x] = psi_i[x] * psi_j[x] for pair r of the chunk.
__global__ void pairform_f64_kernel(const int2 *__restrict__ pairs, int R, const double *__restrict__ psi,
                                    size_t N, double *__restrict__ B) {
    size_t total = (size_t)R * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        size_t r = e / N, x = e % N;
        int2 ij = pairs[r];
        B[e] = psi[(size_t)ij.x * N + x] * psi[(size_t)ij.y * N + x];
    }
}

// Y <- f(Lambda) * Y; block partial of sum_r w_r sum_k f_k Y_k^2 (pair weight w_r =
// multiplicity * g_i * g_j; nullptr weights mean "no energy").
__global__ void scale_f64_kernel(double *__restrict__ Y, int R, size_t N, const double *__restrict__ f,
                                 const int2 *__restrict__ pairs, const double *__restrict__ occ,
                                 double *__restrict__ partial, int want_energy, int scale) {
    double e = 0.0;
    size_t total = (size_t)R * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        size_t r = idx / N, k = idx % N;
        double y = Y[idx];
        double fk = f[k];
        if (want_energy) {
            int2 ij = pairs[r];
            double w = (ij.x == ij.y) ? 1.0 : 2.0;
            if (occ) w *= occ[ij.x] * occ[ij.y];
            e += w * fk * y * y;
        }
        if (scale) Y[idx] = fk * y;
    }
    if (!want_energy) return;
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
        partial[blockIdx.x] = s;
    }
}

// e_x += -1/2 dV * sum(partial[0..n)) in a fixed order (one thread).
__global__ void energy_add_kernel(const double *__restrict__ partial, int n, double factor, double *e_x) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s += partial[b];
        *e_x += factor * s;
    }
}

// (Vx psi)_i -= g_j psi_j phi_ij, (Vx psi)_j -= g_i psi_i phi_ij (i != j), one thread per
// grid point, pairs visited in chunk order (deterministic, no atomics).
__global__ void accum_f64_kernel(const double *__restrict__ phi, const int2 *__restrict__ pairs, int R,
                                 const double *__restrict__ psi, const double *__restrict__ occ, size_t N,
                                 double *__restrict__ vx) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x) {
        for (int r = 0; r < R; ++r) {
            int2 ij = pairs[r];
            double v = phi[(size_t)r * N + x];
            double gi = occ ? occ[ij.x] : 1.0, gj = occ ? occ[ij.y] : 1.0;
            vx[(size_t)ij.x * N + x] -= gj * psi[(size_t)ij.y * N + x] * v;
            if (ij.x != ij.y) vx[(size_t)ij.y * N + x] -= gi * psi[(size_t)ij.x * N + x] * v;
        }
    }
}

int launch_mode(const kx_plan *p, const double *in, double *out, int R, int axis, int inverse, cudaStream_t s) {
    int n = p->n[axis];
    long long inner = axis == 0 ? 1 : (axis == 1 ? p->n[0] : (long long)p->n[0] * p->n[1]);
    long long n_cols = (long long)R * (long long)(p->N / n);
    size_t smem = sizeof(double) * ((size_t)n * n + (size_t)n * (kTQ + 1));
    {
        size_t mx = sizeof(double) * ((size_t)kMaxN * kMaxN + (size_t)kMaxN * (kTQ + 1));
        KX_CUDA_TRY(cudaFuncSetAttribute(mode_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
    }
    long long blocks = (n_cols + kTQ - 1) / kTQ;
    if (int rc = prof_begin(const_cast<kx_plan *>(p), PK_FP64_MODE, s)) return rc;
    mode_f64_kernel<<<(unsigned)blocks, kModeThreads, smem, s>>>(in, out, n_cols, n, inner, p->d_V[axis], inverse);
    KX_LAUNCH_CHECK("mode_f64_kernel launch");
    return prof_end(const_cast<kx_plan *>(p), s);
}

// f(L) on R vectors: forward modes 1, 2, 3; scaling (and energy); inverse modes 3, 2, 1.
// `src` is read, `b0`/`b1` are scratch, the result lands in `dst`.
int fl_chunk(const kx_plan *p, const double *src, double *b0, double *b1, double *dst, int R, bool energy_only,
             const int2 *pairs, const double *occ, double *partial, int n_part, double *e_x, cudaStream_t s) {
    int rc;
    if ((rc = launch_mode(p, src, b0, R, 0, 0, s))) return rc;
    if ((rc = launch_mode(p, b0, b1, R, 1, 0, s))) return rc;
    if ((rc = launch_mode(p, b1, b0, R, 2, 0, s))) return rc;
    const bool want_energy = e_x != nullptr;
    const_cast<kx_plan *>(p)->prof.launches[PK_FP64_OTHER] += want_energy ? 2 : 1;
    const int sblocks = want_energy ? n_part : 4 * p->num_sms;  // grid of the energy partials when summed
    scale_f64_kernel<<<sblocks, 256, 0, s>>>(b0, R, p->N, p->d_f64, pairs, occ, partial, want_energy ? 1 : 0,
                                             energy_only ? 0 : 1);
    KX_LAUNCH_CHECK("scale_f64_kernel launch");
    if (want_energy) {
        energy_add_kernel<<<1, 32, 0, s>>>(partial, n_part, -0.5 * p->dV, e_x);
        KX_LAUNCH_CHECK("energy_add_kernel launch");
    }
    if (energy_only) return KX_OK;
    if ((rc = launch_mode(p, b0, b1, R, 2, 1, s))) return rc;
    if ((rc = launch_mode(p, b1, b0, R, 1, 1, s))) return rc;
    if ((rc = launch_mode(p, b0, dst, R, 0, 1, s))) return rc;
    return KX_OK;
}

long fp64_chunk(const kx_plan *p, long want) {
    const size_t budget = (size_t)2 << 30;  // scratch budget of the float64 path
    long c = (long)std::max<size_t>(1, budget / (3 * p->N * sizeof(double)));
    return std::max(1L, std::min(c, want));
}

}  // namespace

size_t fp64_workspace_bytes(const kx_plan *p, long chunk) {
    return 3 * chunk * p->N * sizeof(double) + 4096 * sizeof(double);
}

int fp64_apply_fL(kx_plan *p, int n_rhs, const double *b, double *x, cudaStream_t s) {
    long chunk = fp64_chunk(p, n_rhs);
    int rc = ensure_workspace(p, fp64_workspace_bytes(p, chunk));
    if (rc) return rc;
    double *w0 = (double *)p->ws.ptr;
    double *w1 = w0 + chunk * p->N;
    for (long c0 = 0; c0 < n_rhs; c0 += chunk) {
        int R = (int)std::min<long>(chunk, n_rhs - c0);
        rc = fl_chunk(p, b + c0 * p->N, w0, w1, x + c0 * p->N, R, false, nullptr, nullptr, nullptr, 0, nullptr, s);
        if (rc) return rc;
    }
    return KX_OK;
}

int fp64_vx(kx_plan *p, int n_orb, const double *psi, const double *occ, double *vx, double *ex,
            bool energy_only, cudaStream_t s, long pair_begin, long pair_end) {
    int rc = ensure_pairs(p, n_orb, s, pair_begin, pair_end);
    if (rc) return rc;
    long P = p->h_group_first.back();  // items of the (range-restricted) pair list
    pair_begin = 0;
    pair_end = P;
    long chunk = fp64_chunk(p, std::max(1L, P));
    rc = ensure_workspace(p, fp64_workspace_bytes(p, chunk));
    if (rc) return rc;
    double *w0 = (double *)p->ws.ptr;
    double *w1 = w0 + chunk * p->N;
    double *w2 = w1 + chunk * p->N;
    double *partial = w2 + chunk * p->N;
    const int n_part = std::min(4096, 4 * p->num_sms);
    if (!energy_only) KX_CUDA_TRY(cudaMemsetAsync(vx, 0, sizeof(double) * n_orb * p->N, s));
    if (ex) KX_CUDA_TRY(cudaMemsetAsync(ex, 0, sizeof(double), s));
    const int2 *pairs = (const int2 *)p->d_pairs;
    for (long c0 = pair_begin; c0 < pair_end; c0 += chunk) {
        int R = (int)std::min<long>(chunk, pair_end - c0);
        int blocks = (int)std::min<size_t>(((size_t)R * p->N + 255) / 256, (size_t)8 * p->num_sms);
        p->prof.launches[PK_FP64_OTHER] += energy_only ? 1 : 2;
        pairform_f64_kernel<<<blocks, 256, 0, s>>>(pairs + c0, R, psi, p->N, w2);
        KX_LAUNCH_CHECK("pairform_f64_kernel launch");
        rc = fl_chunk(p, w2, w0, w1, w2, R, energy_only, pairs + c0, occ, partial, n_part, ex, s);
        if (rc) return rc;
        if (!energy_only) {
            int ab = (int)std::min<size_t>((p->N + 255) / 256, (size_t)8 * p->num_sms);
            accum_f64_kernel<<<ab, 256, 0, s>>>(w2, pairs + c0, R, psi, occ, p->N, vx);
            KX_LAUNCH_CHECK("accum_f64_kernel launch");
        }
    }
    return KX_OK;
}

}  // namespace kx
