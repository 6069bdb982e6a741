// C ABI of kronx: argument checks, plan lifetime, workspaces, dispatch to the
// float64 and tensor-core paths, CUDA-graph batches and the launch-shape tuner.
#include "kx_internal.h"

#include <cmath>
#include <cstdint>
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

namespace kx {

static thread_local int g_last_code = KX_OK;
static thread_local char g_last_msg[512] = "";

int set_error(int code, const std::string &msg) {
    g_last_code = code;
    std::snprintf(g_last_msg, sizeof(g_last_msg), "%s", msg.c_str());
    return code;
}

int cuda_error(cudaError_t e, const char *what) {
    int code = (e == cudaErrorMemoryAllocation) ? KX_ERR_NOMEM : KX_ERR_CUDA;
    return set_error(code, std::string(what) + ": " + cudaGetErrorString(e));
}

// Host-side fault injection for the failure-path tests: KX_FAULT=alloc makes the
// next workspace allocation report KX_ERR_NOMEM without touching the device.
static bool fault_alloc() {
    const char *f = std::getenv("KX_FAULT");
    return f && std::strcmp(f, "alloc") == 0;
}

int ensure_workspace(kx_plan *p, size_t bytes) {
    if (p->ws.bytes >= bytes) return KX_OK;
    if (fault_alloc()) return set_error(KX_ERR_NOMEM, "workspace allocation failed (injected by KX_FAULT=alloc)");
    if (p->ws.ptr) {
        KX_CUDA_TRY(cudaFree(p->ws.ptr));  // implicit device synchronisation
        p->ws.ptr = nullptr;
        p->ws.bytes = 0;
    }
    ++p->config_version;
    cudaError_t e = cudaMalloc(&p->ws.ptr, bytes);
    if (e != cudaSuccess) {
        p->ws.ptr = nullptr;
        return cuda_error(e, "workspace cudaMalloc");
    }
    p->ws.bytes = bytes;
    return KX_OK;
}

// Pair enumeration: orbitals in blocks of kOrbBlock (nb blocks); block pairs
// (I, J), I <= J, first those of the leading columns J < jc column-major
// (J = 0 .. jc-1, I = 0 .. J; jc the fewest columns holding 15% of the block
// pairs), then the rest row-major (I = 0 .. nb-1, J = max(I, jc) .. nb-1);
// inside a diagonal block the upper triangle row-major, inside an off-diagonal
// block all (i, j) row-major.  Each block pair is one accumulation group.  The
// leading columns need only the first orbitals (a host-buffer call starts while
// later orbitals are still being copied); after them the row blocks become
// final one after another (their copies back overlap the rest).  [begin, end)
// restricts the list to a sub-range of this enumeration (groups are cut at the
// range ends).
int leading_columns(int nb) {
    const long long tot = (long long)nb * (nb + 1) / 2, want = (15 * tot + 99) / 100;
    int jc = 1;
    while (jc < nb && (long long)jc * (jc + 1) / 2 < want) ++jc;
    return jc;
}

// With p->blk_mode set, the block pairs of p->blk_req (I <= J each, in the
// given order) are enumerated instead, each whole; begin / end are ignored.
int ensure_pairs(kx_plan *p, int n_orb, cudaStream_t s, long long begin, long long end) {
    (void)s;
    const long long P_all = (long long)n_orb * (n_orb + 1) / 2;
    if (end < 0) end = P_all;
    if (p->blk_mode) {
        begin = 0;
        end = P_all;
        if (p->ws_norb == n_orb && p->blk_cur == p->blk_req) return KX_OK;
    } else if (p->ws_norb == n_orb && p->blk_cur.empty() && p->pr_begin == begin && p->pr_end == end) {
        return KX_OK;
    }
    ++p->config_version;  // the list is rebuilt in place
    std::vector<int> pairs, slots;
    std::vector<Group> groups;
    std::vector<int> first;
    std::vector<unsigned char> mask((size_t)n_orb * n_orb, 0);
    pairs.reserve(2 * (size_t)(end - begin));
    slots.reserve(2 * (size_t)(end - begin));
    const int nb = (n_orb + kOrbBlock - 1) / kOrbBlock;
    // the block pairs to visit: all (I <= J) in the order above, or the explicit list
    std::vector<int> visit;
    if (p->blk_mode) {
        visit = p->blk_req;
    } else {
        visit.reserve((size_t)nb * (nb + 1));
        const int jc = leading_columns(nb);
        for (int JB = 0; JB < jc; ++JB)
            for (int IB = 0; IB <= JB; ++IB) {
                visit.push_back(IB);
                visit.push_back(JB);
            }
        for (int IB = 0; IB < nb; ++IB)
            for (int JB = std::max(IB, jc); JB < nb; ++JB) {
                visit.push_back(IB);
                visit.push_back(JB);
            }
    }
    long long k = 0;
    for (size_t v = 0; v + 1 < visit.size(); v += 2) {
        {
            const int IB = visit[v], JB = visit[v + 1];
            const int I0 = IB * kOrbBlock, bi = std::min(kOrbBlock, n_orb - I0);
            const int J0 = JB * kOrbBlock, bj = std::min(kOrbBlock, n_orb - J0);
            Group g{};
            g.first_item = (int)(pairs.size() / 2);
            g.n_items = 0;
            g.n_slots = (IB == JB) ? bi : bi + bj;
            for (int t = 0; t < bi; ++t) g.orb[t] = I0 + t;
            if (IB != JB)
                for (int t = 0; t < bj; ++t) g.orb[bi + t] = J0 + t;
            for (int si = 0; si < bi; ++si) {
                for (int sj = (IB == JB ? si : 0); sj < (IB == JB ? bi : bj); ++sj, ++k) {
                    if (k < begin || k >= end) continue;
                    const int oi = I0 + si, oj = (IB == JB ? I0 : J0) + sj;
                    mask[(size_t)oi * n_orb + oj] = mask[(size_t)oj * n_orb + oi] = 1;
                    pairs.push_back(I0 + si);
                    pairs.push_back((IB == JB ? I0 : J0) + sj);
                    slots.push_back(si);
                    slots.push_back(IB == JB ? sj : bi + sj);
                    ++g.n_items;
                }
            }
            if (g.n_items > 0) {
                groups.push_back(g);
                first.push_back(g.first_item);
            }
        }
    }
    first.push_back((int)(pairs.size() / 2));
    std::vector<int> last(n_orb, -1), maxorb(groups.size(), 0);
    for (size_t gi = 0; gi < groups.size(); ++gi)
        for (int t = 0; t < groups[gi].n_slots; ++t) {
            last[groups[gi].orb[t]] = (int)gi;
            maxorb[gi] = std::max(maxorb[gi], groups[gi].orb[t]);
        }
    const size_t P = pairs.size() / 2;
    if (P > p->pairs_cap) {
        cudaFree(p->d_pairs);
        cudaFree(p->d_item_slot);
        p->d_pairs = p->d_item_slot = nullptr;
        p->pairs_cap = 0;
        cudaError_t e = cudaMalloc(&p->d_pairs, sizeof(int) * 2 * std::max<size_t>(P, 1));
        if (e == cudaSuccess) e = cudaMalloc(&p->d_item_slot, sizeof(int) * 2 * std::max<size_t>(P, 1));
        if (e != cudaSuccess) return cuda_error(e, "pair list cudaMalloc");
        p->pairs_cap = P;
    }
    if (groups.size() > p->groups_cap) {
        cudaFree(p->d_groups);
        p->d_groups = nullptr;
        p->groups_cap = 0;
        cudaError_t e = cudaMalloc(&p->d_groups, sizeof(Group) * groups.size());
        if (e != cudaSuccess) return cuda_error(e, "group table cudaMalloc");
        p->groups_cap = groups.size();
    }
    if (mask.size() > p->pair_mask_cap) {
        cudaFree(p->d_pair_mask);
        p->d_pair_mask = nullptr;
        p->pair_mask_cap = 0;
        cudaError_t e = cudaMalloc(&p->d_pair_mask, mask.size());
        if (e != cudaSuccess) return cuda_error(e, "pair mask cudaMalloc");
        p->pair_mask_cap = mask.size();
    }
    KX_CUDA_TRY(cudaMemcpy(p->d_pair_mask, mask.data(), mask.size(), cudaMemcpyHostToDevice));
    if (P) {
        KX_CUDA_TRY(cudaMemcpy(p->d_pairs, pairs.data(), sizeof(int) * 2 * P, cudaMemcpyHostToDevice));
        KX_CUDA_TRY(cudaMemcpy(p->d_item_slot, slots.data(), sizeof(int) * 2 * P, cudaMemcpyHostToDevice));
        KX_CUDA_TRY(cudaMemcpy(p->d_groups, groups.data(), sizeof(Group) * groups.size(), cudaMemcpyHostToDevice));
    }
    p->h_group_first = first;
    p->h_orb_last = last;
    p->h_group_maxorb = maxorb;
    p->ws_norb = n_orb;
    p->pr_begin = begin;
    p->pr_end = end;
    if (p->blk_mode)
        p->blk_cur = p->blk_req;
    else
        p->blk_cur.clear();
    return KX_OK;
}

static int prof_event(kx_plan *p, cudaEvent_t *out) {
    Profiler &P = p->prof;
    if (P.used == P.pool.size()) {
        cudaEvent_t e;
        KX_CUDA_TRY(cudaEventCreate(&e));
        P.pool.push_back(e);
    }
    *out = P.pool[P.used++];
    return KX_OK;
}

int prof_begin(kx_plan *p, int kind, cudaStream_t s) {
    p->prof.launches[kind] += 1;
    if (!p->prof.on) return KX_OK;
    cudaEvent_t e;
    if (int rc = prof_event(p, &e)) return rc;
    p->prof.marks.push_back({kind, p->prof.used - 1});
    KX_CUDA_TRY(cudaEventRecord(e, s));
    return KX_OK;
}

int prof_end(kx_plan *p, cudaStream_t s) {
    if (!p->prof.on) return KX_OK;
    cudaEvent_t e;
    if (int rc = prof_event(p, &e)) return rc;
    KX_CUDA_TRY(cudaEventRecord(e, s));
    return KX_OK;
}

static int reserve(kx_plan *p, int n_orb) {
    int rc = ensure_pairs(p, n_orb, nullptr);
    if (rc) return rc;
    if ((rc = mp_reserve(p, n_orb))) return rc;
    if (p->precision == KX_FP64) {
        const long P = (long)n_orb * (n_orb + 1) / 2;
        const size_t budget = (size_t)2 << 30;
        long c = (long)std::max<size_t>(1, budget / (3 * p->N * sizeof(double)));
        return ensure_workspace(p, fp64_workspace_bytes(p, std::min(c, P)));
    }
    const long P = (long)n_orb * (n_orb + 1) / 2;
    const long chunk = std::min<long>(tc_default_chunk(p, n_orb), P);
    return ensure_workspace(p, tc_workspace_bytes(p, n_orb, chunk));
}

static int dispatch_vx(kx_plan *p, int n_orb, const double *psi, const double *occ, double *vx, double *ex,
                       bool energy_only, cudaStream_t s, long pair_begin = 0, long pair_end = -1) {
    p->mp_applied = false;
    int rc = p->precision == KX_FP64 ? fp64_vx(p, n_orb, psi, occ, vx, ex, energy_only, s, pair_begin, pair_end)
                                     : tc_vx(p, n_orb, psi, occ, vx, ex, energy_only, s, pair_begin, pair_end);
    // boundary values from the multipole expansion: the rank-K correction of
    // the same pair range (its mask was built by the solve's ensure_pairs),
    // unless the split path already started its accumulator from it
    if (!rc && p->mp_lmax >= 0 && !p->mp_applied) rc = mp_correct_vx(p, n_orb, psi, occ, vx, ex, energy_only, s);
    p->mp_applied = false;
    return rc;
}

static int check_plan(const kx_plan *p) {
    if (!p) return set_error(KX_ERR_ARG, "plan is NULL");
    return KX_OK;
}

// Launch shapes chosen by kx_autotune, kept for the life of the process and
// keyed by what the kernels' launch shapes depend on (grid, precision, device
// model and orbital count), so that later plans of the same shape start tuned.
static std::mutex g_tune_mu;
static std::map<std::string, TuneParams> g_tune_table;

static std::string tune_key(const kx_plan *p, int n_orb) {
    char name[256] = "";
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) std::snprintf(name, sizeof(name), "%s", prop.name);
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%d,%d,%d|%d|%d|%s", p->n[0], p->n[1], p->n[2], p->precision, n_orb, name);
    return buf;
}

static bool tune_lookup(kx_plan *p, int n_orb) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_table.find(tune_key(p, n_orb));
    if (it == g_tune_table.end()) return false;
    p->tune = it->second;
    return true;
}

static void tune_store(const kx_plan *p, int n_orb) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_table[tune_key(p, n_orb)] = p->tune;
}

}  // namespace kx

using namespace kx;

struct kx_batch_s {
    std::vector<kx_plan *> plans;
    std::vector<int> n_orb;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const double *> last_psi;
    std::vector<double *> last_vx;
    double *last_ex = nullptr;
    std::vector<unsigned long long> versions;  // plans' config_version at capture
    int device = 0;
};

extern "C" {

const char *kx_strerror(int code) {
    switch (code) {
        case KX_OK: return "KX_OK";
        case KX_ERR_ARG: return "KX_ERR_ARG";
        case KX_ERR_SINGULAR: return "KX_ERR_SINGULAR";
        case KX_ERR_NOMEM: return "KX_ERR_NOMEM";
        case KX_ERR_CUDA: return "KX_ERR_CUDA";
        case KX_ERR_TIMEOUT: return "KX_ERR_TIMEOUT";
        case KX_ERR_UNSUPPORTED: return "KX_ERR_UNSUPPORTED";
        default: return "KX_ERR_UNKNOWN";
    }
}

int kx_last_error_detail(char *buf, int len) {
    if (buf && len > 0) std::snprintf(buf, (size_t)len, "%s", g_last_msg);
    return g_last_code;
}

int kx_plan_create(const kx_grid *grid, const kx_kernel *kernel, int precision, kx_plan **out) {
    if (!grid || !kernel || !out) return set_error(KX_ERR_ARG, "kx_plan_create: NULL argument");
    *out = nullptr;
    for (int a = 0; a < 3; ++a) {
        if (grid->n[a] < 2) return set_error(KX_ERR_ARG, "kx_plan_create: n[a] must be >= 2");
        if (grid->n[a] > kMaxN) return set_error(KX_ERR_UNSUPPORTED, "kx_plan_create: n[a] > 128");
        if (!(grid->h[a] > 0.0)) return set_error(KX_ERR_ARG, "kx_plan_create: h[a] must be > 0");
        if (grid->bc[a] != KX_DIRICHLET && grid->bc[a] != KX_PERIODIC)
            return set_error(KX_ERR_ARG, "kx_plan_create: bc[a] must be KX_DIRICHLET or KX_PERIODIC");
    }
    if (grid->fd_order < 2 || grid->fd_order % 2 || grid->fd_order > 24)
        return set_error(KX_ERR_ARG, "kx_plan_create: fd_order must be even, 2..24");
    if (kernel->kind != KX_UNSCREENED && kernel->kind != KX_SCREENED)
        return set_error(KX_ERR_ARG, "kx_plan_create: unknown kernel kind");
    if (kernel->kind == KX_SCREENED && !(kernel->omega > 0.0))
        return set_error(KX_ERR_ARG, "kx_plan_create: omega must be > 0 for the screened kernel");
    if (precision != KX_FP64 && precision != KX_F16X3 && precision != KX_FFT32)
        return set_error(KX_ERR_ARG, "kx_plan_create: unknown precision");
    if (precision == KX_FFT32 && !fft_supported(grid->n, grid->bc))
        return set_error(KX_ERR_UNSUPPORTED,
                         "kx_plan_create: KX_FFT32 needs periodic axes whose sizes are products of 2, 3 and 5 "
                         "and an n[0] x n[1] plane of at most about 12,000 points");
    if (precision == KX_F16X3)
        for (int a = 0; a < 3; ++a)
            if (grid->n[a] % 8)
                return set_error(KX_ERR_UNSUPPORTED, "kx_plan_create: KX_F16X3 needs n[a] % 8 == 0");
    if (kernel->kind == KX_UNSCREENED && grid->bc[0] == KX_PERIODIC && grid->bc[1] == KX_PERIODIC &&
        grid->bc[2] == KX_PERIODIC)
        return set_error(KX_ERR_SINGULAR, "kx_plan_create: unscreened kernel with all axes periodic is singular");

    kx_plan *p = new (std::nothrow) kx_plan_s();
    if (!p) return set_error(KX_ERR_NOMEM, "kx_plan_create: host allocation failed");
    for (int a = 0; a < 3; ++a) {
        p->n[a] = grid->n[a];
        p->h[a] = grid->h[a];
        p->bc[a] = grid->bc[a];
        p->np[a] = round_up(grid->n[a], 16);
    }
    p->fd_order = grid->fd_order;
    p->kind = kernel->kind;
    p->omega = kernel->omega;
    p->precision = precision;
    p->N = (size_t)p->n[0] * p->n[1] * p->n[2];
    p->dV = p->h[0] * p->h[1] * p->h[2];
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_error(e, "kx_plan_create: no usable CUDA device");
    }
    int rc = plan_setup(p);
    if (rc) {
        plan_free(p);
        delete p;
        return rc;
    }
    *out = p;
    return KX_OK;
}

int kx_plan_destroy(kx_plan *plan) {
    if (!plan) return KX_OK;
    cudaSetDevice(plan->device);
    cudaDeviceSynchronize();
    plan_free(plan);
    delete plan;
    return KX_OK;
}

int kx_plan_eig(const kx_plan *plan, int axis, double *lam, double *V) {
    if (int rc = check_plan(plan)) return rc;
    if (axis < 0 || axis > 2) return set_error(KX_ERR_ARG, "kx_plan_eig: axis must be 0, 1 or 2");
    const int n = plan->n[axis];
    if (lam) KX_CUDA_TRY(cudaMemcpy(lam, plan->d_lam[axis], sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (V) KX_CUDA_TRY(cudaMemcpy(V, plan->d_V[axis], sizeof(double) * n * n, cudaMemcpyDeviceToHost));
    return KX_OK;
}

int kx_plan_ftable(const kx_plan *plan, double *f) {
    if (int rc = check_plan(plan)) return rc;
    if (!f) return set_error(KX_ERR_ARG, "kx_plan_ftable: NULL output");
    KX_CUDA_TRY(cudaMemcpy(f, plan->d_f64, sizeof(double) * plan->N, cudaMemcpyDeviceToHost));
    return KX_OK;
}

int kx_apply_fL(kx_plan *plan, int n_rhs, const double *b, double *x, kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (n_rhs < 0) return set_error(KX_ERR_ARG, "kx_apply_fL: n_rhs < 0");
    if (n_rhs == 0) return KX_OK;
    if (!b || !x) return set_error(KX_ERR_ARG, "kx_apply_fL: NULL buffer");
    if (b == x) return set_error(KX_ERR_ARG, "kx_apply_fL: x must not overlap b");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int rc = plan->precision == KX_FP64 ? fp64_apply_fL(plan, n_rhs, b, x, s) : tc_apply_fL(plan, n_rhs, b, x, s);
    if (!rc && plan->mp_lmax >= 0) rc = mp_correct_apply(plan, n_rhs, b, x, s);
    return rc;
}

int kx_apply_fL_noalloc(kx_plan *plan, int n_rhs, const double *b, double *x, kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (n_rhs < 0) return set_error(KX_ERR_ARG, "kx_apply_fL_noalloc: n_rhs < 0");
    if (n_rhs == 0) return KX_OK;
    if (!b || !x) return set_error(KX_ERR_ARG, "kx_apply_fL_noalloc: NULL buffer");
    if (b == x) return set_error(KX_ERR_ARG, "kx_apply_fL_noalloc: x must not overlap b");
    if (plan->mp_lmax >= 0)
        return set_error(KX_ERR_UNSUPPORTED, "kx_apply_fL_noalloc: not available with multipole boundary values");
    if (plan->precision == KX_FFT32)
        return set_error(KX_ERR_UNSUPPORTED, "kx_apply_fL_noalloc: not available on KX_FFT32 plans");
    return tc_apply_fL_noalloc(plan, n_rhs, b, x, reinterpret_cast<cudaStream_t>(stream));
}

int kx_vx_apply(kx_plan *plan, int n_orb, const double *psi, const double *occ, double *vx_psi, double *e_x,
                kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (n_orb < 1 || n_orb > 4096) return set_error(KX_ERR_ARG, "kx_vx_apply: n_orb must be in 1..4096");
    if (!psi || !vx_psi) return set_error(KX_ERR_ARG, "kx_vx_apply: NULL buffer");
    if (psi == vx_psi) return set_error(KX_ERR_ARG, "kx_vx_apply: vx_psi must not overlap psi");
    return dispatch_vx(plan, n_orb, psi, occ, vx_psi, e_x, false, reinterpret_cast<cudaStream_t>(stream));
}

int kx_vx_apply_pairs(kx_plan *plan, int n_orb, const double *psi, const double *occ, long long pair_begin,
                      long long pair_end, double *vx_psi, double *e_x, kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (n_orb < 1 || n_orb > 4096) return set_error(KX_ERR_ARG, "kx_vx_apply_pairs: n_orb must be in 1..4096");
    const long long P = (long long)n_orb * (n_orb + 1) / 2;
    if (pair_begin < 0 || pair_end < pair_begin || pair_end > P)
        return set_error(KX_ERR_ARG, "kx_vx_apply_pairs: need 0 <= pair_begin <= pair_end <= n_orb(n_orb+1)/2");
    if (!psi || !vx_psi) return set_error(KX_ERR_ARG, "kx_vx_apply_pairs: NULL buffer");
    if (psi == vx_psi) return set_error(KX_ERR_ARG, "kx_vx_apply_pairs: vx_psi must not overlap psi");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (pair_end == pair_begin) {
        KX_CUDA_TRY(cudaMemsetAsync(vx_psi, 0, sizeof(double) * (size_t)n_orb * plan->N, s));
        if (e_x) KX_CUDA_TRY(cudaMemsetAsync(e_x, 0, sizeof(double), s));
        return KX_OK;
    }
    return dispatch_vx(plan, n_orb, psi, occ, vx_psi, e_x, false, s, (long)pair_begin, (long)pair_end);
}

int kx_vx_apply_block_pairs(kx_plan *plan, int n_orb, const double *psi, const double *occ, const int *blocks,
                            int n_blocks, double *vx_psi, double *e_x, kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (n_orb < 1 || n_orb > 4096) return set_error(KX_ERR_ARG, "kx_vx_apply_block_pairs: n_orb must be in 1..4096");
    if (!psi || !vx_psi) return set_error(KX_ERR_ARG, "kx_vx_apply_block_pairs: NULL buffer");
    if (psi == vx_psi) return set_error(KX_ERR_ARG, "kx_vx_apply_block_pairs: vx_psi must not overlap psi");
    const int nb = (n_orb + kOrbBlock - 1) / kOrbBlock;
    if (n_blocks < 0 || n_blocks > nb * (nb + 1) / 2 || (n_blocks > 0 && !blocks))
        return set_error(KX_ERR_ARG, "kx_vx_apply_block_pairs: need 0 <= n_blocks <= nb (nb + 1) / 2 and a list");
    std::vector<int> req(blocks, blocks + 2 * (size_t)n_blocks);
    std::vector<unsigned char> seen((size_t)nb * nb, 0);
    for (int b = 0; b < n_blocks; ++b) {
        const int I = req[2 * b], J = req[2 * b + 1];
        if (I < 0 || J < I || J >= nb)
            return set_error(KX_ERR_ARG, "kx_vx_apply_block_pairs: each block pair needs 0 <= I <= J < ceil(n_orb / 4)");
        if (seen[(size_t)I * nb + J]++)
            return set_error(KX_ERR_ARG, "kx_vx_apply_block_pairs: a block pair appears twice");
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (n_blocks == 0) {
        KX_CUDA_TRY(cudaMemsetAsync(vx_psi, 0, sizeof(double) * (size_t)n_orb * plan->N, s));
        if (e_x) KX_CUDA_TRY(cudaMemsetAsync(e_x, 0, sizeof(double), s));
        return KX_OK;
    }
    plan->blk_req.swap(req);
    plan->blk_mode = true;
    int rc = dispatch_vx(plan, n_orb, psi, occ, vx_psi, e_x, false, s);
    plan->blk_mode = false;
    return rc;
}

int kx_energy(kx_plan *plan, int n_orb, const double *psi, const double *occ, double *e_x, kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (n_orb < 1 || n_orb > 4096) return set_error(KX_ERR_ARG, "kx_energy: n_orb must be in 1..4096");
    if (!psi || !e_x) return set_error(KX_ERR_ARG, "kx_energy: NULL buffer");
    return dispatch_vx(plan, n_orb, psi, occ, nullptr, e_x, true, reinterpret_cast<cudaStream_t>(stream));
}

int kx_vx_apply_host(kx_plan *plan, int n_orb, const double *psi, const double *occ, double *vx_psi, double *e_x,
                     kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (n_orb < 1 || n_orb > 4096) return set_error(KX_ERR_ARG, "kx_vx_apply_host: n_orb must be in 1..4096");
    if (!psi || !vx_psi) return set_error(KX_ERR_ARG, "kx_vx_apply_host: NULL buffer");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t vec = sizeof(double) * (size_t)n_orb * plan->N;
    const size_t need = 2 * vec + sizeof(double) * (n_orb + 1) + 512;
    if (plan->ws_host.bytes < need) {
        if (fault_alloc()) return set_error(KX_ERR_NOMEM, "staging allocation failed (injected by KX_FAULT=alloc)");
        cudaFree(plan->ws_host.ptr);
        plan->ws_host.ptr = nullptr;
        plan->ws_host.bytes = 0;
        cudaError_t e = cudaMalloc(&plan->ws_host.ptr, need);
        if (e != cudaSuccess) return cuda_error(e, "kx_vx_apply_host staging cudaMalloc");
        plan->ws_host.bytes = need;
    }
    if (!plan->copy_stream) KX_CUDA_TRY(cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking));
    double *d_psi = (double *)plan->ws_host.ptr;
    double *d_vx = d_psi + (size_t)n_orb * plan->N;
    double *d_ex = d_vx + (size_t)n_orb * plan->N;
    double *d_occ = occ ? d_ex + 1 : nullptr;
    if (occ) KX_CUDA_TRY(cudaMemcpyAsync(d_occ, occ, sizeof(double) * n_orb, cudaMemcpyHostToDevice, s));
    // The orbitals go over in pieces of whole orbital blocks on their own stream
    // (after the work already queued on s), each with an event; the split path
    // starts on the first pieces while the later ones are still copying (its
    // pair order needs the first orbitals first).  Float64 plans and plans with
    // multipole boundary values take the orbitals in one copy first.
    const char *pe = std::getenv("KX_HOST_PIECES");  // 0: one copy first (comparison runs)
    const bool by_pieces = plan->precision != KX_FP64 && plan->mp_lmax < 0 && !(pe && std::atoi(pe) == 0);
    if (by_pieces) {
        if (!plan->h2d_stream) KX_CUDA_TRY(cudaStreamCreateWithFlags(&plan->h2d_stream, cudaStreamNonBlocking));
        const int nb = (n_orb + kOrbBlock - 1) / kOrbBlock;
        const int n_pieces = std::min(8, nb);
        const int bpp = (nb + n_pieces - 1) / n_pieces;  // blocks per piece
        InputPieces pcs;
        for (int b0 = 0; b0 < nb; b0 += bpp) pcs.end.push_back(std::min(n_orb, (b0 + bpp) * kOrbBlock));
        while (plan->h2d_events.size() < pcs.end.size() + 1) {
            cudaEvent_t ev;
            KX_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            plan->h2d_events.push_back(ev);
        }
        cudaEvent_t start = plan->h2d_events.back();
        KX_CUDA_TRY(cudaEventRecord(start, s));
        KX_CUDA_TRY(cudaStreamWaitEvent(plan->h2d_stream, start, 0));
        int o0 = 0;
        for (size_t k = 0; k < pcs.end.size(); ++k) {
            const int o1 = pcs.end[k];
            KX_CUDA_TRY(cudaMemcpyAsync(d_psi + (size_t)o0 * plan->N, psi + (size_t)o0 * plan->N,
                                        sizeof(double) * (size_t)(o1 - o0) * plan->N, cudaMemcpyHostToDevice,
                                        plan->h2d_stream));
            KX_CUDA_TRY(cudaEventRecord(plan->h2d_events[k], plan->h2d_stream));
            pcs.ready.push_back(plan->h2d_events[k]);
            o0 = o1;
        }
        plan->in_pieces = pcs;
    } else {
        KX_CUDA_TRY(cudaMemcpyAsync(d_psi, psi, vec, cudaMemcpyHostToDevice, s));
    }
    // rows of Vx psi that the split path reports final are copied back on the
    // plan's copy stream while the later chunks compute
    struct Ctx {
        kx_plan *p;
        double *host;
        const double *dev;
        size_t N;
        int copied, events, rc;
    } ctx{plan, vx_psi, d_vx, plan->N, 0, 0, KX_OK};
    plan->final_hook.ctx = &ctx;
    plan->final_hook.fn = [](void *c, int o0, int o1, cudaStream_t st) {
        Ctx *x = static_cast<Ctx *>(c);
        if (x->rc || o1 <= o0) return;
        kx_plan *p = x->p;
        if ((size_t)x->events == p->copy_events.size()) {
            cudaEvent_t ev;
            cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) {
                x->rc = cuda_error(e, "kx_vx_apply_host copy event");
                return;
            }
            p->copy_events.push_back(ev);
        }
        cudaEvent_t ev = p->copy_events[x->events++];
        cudaError_t e = cudaEventRecord(ev, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->copy_stream, ev, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(x->host + (size_t)o0 * x->N, x->dev + (size_t)o0 * x->N,
                                sizeof(double) * (size_t)(o1 - o0) * x->N, cudaMemcpyDeviceToHost, p->copy_stream);
        if (e != cudaSuccess) x->rc = cuda_error(e, "kx_vx_apply_host row copy");
        x->copied = o1;
    };
    // with multipole boundary values every row changes after the pair loop: no early copies
    if (plan->mp_lmax >= 0) plan->final_hook = FinalHook{};
    int rc = dispatch_vx(plan, n_orb, d_psi, d_occ, d_vx, d_ex, false, s);
    plan->final_hook = FinalHook{};
    plan->in_pieces = InputPieces{};
    if (!rc) rc = ctx.rc;
    // the copy stream's work joins the caller's stream before the rest is read
    cudaEvent_t done;
    KX_CUDA_TRY(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(done, plan->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, done, 0);
    cudaEventDestroy(done);
    if (e != cudaSuccess) return cuda_error(e, "kx_vx_apply_host copy join");
    if (rc) {
        cudaStreamSynchronize(s);
        if (plan->h2d_stream) cudaStreamSynchronize(plan->h2d_stream);  // the caller's psi is read until then
        return rc;
    }
    if (ctx.copied < n_orb)
        KX_CUDA_TRY(cudaMemcpyAsync(vx_psi + (size_t)ctx.copied * plan->N, d_vx + (size_t)ctx.copied * plan->N,
                                    sizeof(double) * (size_t)(n_orb - ctx.copied) * plan->N, cudaMemcpyDeviceToHost, s));
    if (e_x) KX_CUDA_TRY(cudaMemcpyAsync(e_x, d_ex, sizeof(double), cudaMemcpyDeviceToHost, s));
    KX_CUDA_TRY(cudaStreamSynchronize(s));
    return KX_OK;
}

int kx_ace(kx_plan *plan, int n_orb, const double *psi, const double *vx_psi, double *xi, double *M_out,
           kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (n_orb < 1 || n_orb > 256) return set_error(KX_ERR_ARG, "kx_ace: n_orb must be in 1..256");
    if (!psi || !vx_psi || !xi) return set_error(KX_ERR_ARG, "kx_ace: NULL buffer");
    if (xi == psi || xi == vx_psi) return set_error(KX_ERR_ARG, "kx_ace: xi must not overlap the inputs");
    return ace_run(plan, n_orb, psi, vx_psi, xi, M_out, reinterpret_cast<cudaStream_t>(stream));
}

int kx_ace_apply(kx_plan *plan, int n_xi, const double *xi, int n_vec, const double *phi, double *out,
                 kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (n_xi < 1 || n_xi > 256) return set_error(KX_ERR_ARG, "kx_ace_apply: n_xi must be in 1..256");
    if (n_vec < 1) return set_error(KX_ERR_ARG, "kx_ace_apply: n_vec must be >= 1");
    if (!xi || !phi || !out) return set_error(KX_ERR_ARG, "kx_ace_apply: NULL buffer");
    const size_t N = plan->N;
    auto overlaps = [N](const double *a, size_t na, const double *b, size_t nb) {
        return a < b + nb * N && b < a + na * N;
    };
    if (overlaps(out, (size_t)n_vec, xi, (size_t)n_xi) || overlaps(out, (size_t)n_vec, phi, (size_t)n_vec))
        return set_error(KX_ERR_ARG, "kx_ace_apply: out must not overlap xi or phi");
    return ace_apply_run(plan, n_xi, xi, n_vec, phi, out, reinterpret_cast<cudaStream_t>(stream));
}

namespace {
int check_kpoints(kx_plan *plan, const char *fn, int n_kpt, const double *theta, const double *wk, int n_orb,
                  const double *psi) {
    if (n_kpt < 1 || n_kpt > 1024) return set_error(KX_ERR_ARG, std::string(fn) + ": n_kpt must be in 1..1024");
    if (n_orb < 1 || n_orb > 4096) return set_error(KX_ERR_ARG, std::string(fn) + ": n_orb must be in 1..4096");
    if (!theta || !wk || !psi) return set_error(KX_ERR_ARG, std::string(fn) + ": NULL argument");
    for (int i = 0; i < 3 * n_kpt; ++i)
        if (!std::isfinite(theta[i])) return set_error(KX_ERR_ARG, std::string(fn) + ": non-finite phase");
    for (int i = 0; i < n_kpt; ++i)
        if (!std::isfinite(wk[i])) return set_error(KX_ERR_ARG, std::string(fn) + ": non-finite weight");
    if (plan->mp_lmax >= 0)
        return set_error(KX_ERR_UNSUPPORTED, std::string(fn) + ": plans with multipole boundary values are isolated");
    return KX_OK;
}
bool misaligned16(const void *p) { return reinterpret_cast<uintptr_t>(p) % 16 != 0; }
}  // namespace

int kx_vx_apply_kpoint(kx_plan *plan, int n_kpt, const double *theta, const double *wk, int n_orb,
                       const double *psi, const double *occ, int k_index, int n_vec, const double *phi,
                       double *out, kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (int rc = check_kpoints(plan, "kx_vx_apply_kpoint", n_kpt, theta, wk, n_orb, psi)) return rc;
    if (k_index < 0 || k_index >= n_kpt) return set_error(KX_ERR_ARG, "kx_vx_apply_kpoint: k_index out of range");
    if (n_vec < 1 || n_vec > 4096) return set_error(KX_ERR_ARG, "kx_vx_apply_kpoint: n_vec must be in 1..4096");
    if (!phi || !out) return set_error(KX_ERR_ARG, "kx_vx_apply_kpoint: NULL buffer");
    if (misaligned16(psi) || misaligned16(phi) || misaligned16(out))
        return set_error(KX_ERR_ARG, "kx_vx_apply_kpoint: complex buffers must be 16-byte aligned");
    const size_t c = 2 * plan->N;
    auto overlaps = [](const double *a, size_t na, const double *b, size_t nb) { return a < b + nb && b < a + na; };
    if (overlaps(out, c * n_vec, psi, c * n_orb * (size_t)n_kpt) || overlaps(out, c * n_vec, phi, c * n_vec))
        return set_error(KX_ERR_ARG, "kx_vx_apply_kpoint: out must not overlap psi or phi");
    return bloch_vx_apply(plan, n_kpt, theta, wk, n_orb, psi, occ, k_index, n_vec, phi, out,
                          reinterpret_cast<cudaStream_t>(stream));
}

int kx_vx_kpoints(kx_plan *plan, int n_kpt, const double *theta, const double *wk, int n_orb, const double *psi,
                  const double *occ, double *vx, double *ex, kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (int rc = check_kpoints(plan, "kx_vx_kpoints", n_kpt, theta, wk, n_orb, psi)) return rc;
    if (!vx) return set_error(KX_ERR_ARG, "kx_vx_kpoints: NULL buffer");
    if (misaligned16(psi) || misaligned16(vx))
        return set_error(KX_ERR_ARG, "kx_vx_kpoints: complex buffers must be 16-byte aligned");
    const size_t c = 2 * plan->N * (size_t)n_orb * n_kpt;
    if (vx < psi + c && psi < vx + c) return set_error(KX_ERR_ARG, "kx_vx_kpoints: vx must not overlap psi");
    return bloch_vx_all(plan, n_kpt, theta, wk, n_orb, psi, occ, 0, (long long)n_kpt * (n_kpt + 1) / 2, vx, ex,
                        reinterpret_cast<cudaStream_t>(stream));
}

int kx_vx_kpoint_blocks(kx_plan *plan, int n_kpt, const double *theta, const double *wk, int n_orb,
                        const double *psi, const double *occ, long long block_begin, long long block_end, double *vx,
                        double *ex, kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (int rc = check_kpoints(plan, "kx_vx_kpoint_blocks", n_kpt, theta, wk, n_orb, psi)) return rc;
    const long long B = (long long)n_kpt * (n_kpt + 1) / 2;
    if (block_begin < 0 || block_end > B || block_begin > block_end)
        return set_error(KX_ERR_ARG, "kx_vx_kpoint_blocks: need 0 <= block_begin <= block_end <= n_kpt (n_kpt + 1) / 2");
    if (!vx) return set_error(KX_ERR_ARG, "kx_vx_kpoint_blocks: NULL buffer");
    if (misaligned16(psi) || misaligned16(vx))
        return set_error(KX_ERR_ARG, "kx_vx_kpoint_blocks: complex buffers must be 16-byte aligned");
    const size_t c = 2 * plan->N * (size_t)n_orb * n_kpt;
    if (vx < psi + c && psi < vx + c) return set_error(KX_ERR_ARG, "kx_vx_kpoint_blocks: vx must not overlap psi");
    return bloch_vx_all(plan, n_kpt, theta, wk, n_orb, psi, occ, block_begin, block_end, vx, ex,
                        reinterpret_cast<cudaStream_t>(stream));
}

int kx_energy_kpoints(kx_plan *plan, int n_kpt, const double *theta, const double *wk, int n_orb,
                      const double *psi, const double *occ, double *ex, kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (int rc = check_kpoints(plan, "kx_energy_kpoints", n_kpt, theta, wk, n_orb, psi)) return rc;
    if (!ex) return set_error(KX_ERR_ARG, "kx_energy_kpoints: NULL ex");
    if (misaligned16(psi)) return set_error(KX_ERR_ARG, "kx_energy_kpoints: psi must be 16-byte aligned");
    return bloch_energy(plan, n_kpt, theta, wk, n_orb, psi, occ, ex, reinterpret_cast<cudaStream_t>(stream));
}

namespace kx {
namespace {
// grad[a][x] = 2 dV g_a G[a][x] in place
__global__ void grad_scale_kernel(double *__restrict__ g, const double *__restrict__ occ, int n, long long N,
                                  double two_dv) {
    const long long total = (long long)n * N;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        g[e] *= two_dv * (occ ? occ[e / N] : 1.0);
}
}  // namespace
}  // namespace kx

int kx_energy_gradient(kx_plan *plan, int n_orb, const double *psi, const double *occ, double *grad, double *e_x,
                       kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (n_orb < 1 || n_orb > 4096) return set_error(KX_ERR_ARG, "kx_energy_gradient: n_orb must be in 1..4096");
    if (!psi || !grad) return set_error(KX_ERR_ARG, "kx_energy_gradient: NULL buffer");
    if (psi == grad) return set_error(KX_ERR_ARG, "kx_energy_gradient: grad must not overlap psi");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // G = Vx psi, with the multipole correction in its symmetric form when it is on
    plan->mp_grad = plan->mp_lmax >= 0;
    int rc = dispatch_vx(plan, n_orb, psi, occ, grad, e_x, false, s);
    plan->mp_grad = false;
    if (rc) return rc;
    grad_scale_kernel<<<4 * plan->num_sms, 256, 0, s>>>(grad, occ, n_orb, (long long)plan->N, 2.0 * plan->dV);
    KX_LAUNCH_CHECK("grad_scale_kernel launch");
    return KX_OK;
}

int kx_plan_set_multipole(kx_plan *plan, int l_max) {
    if (int rc = check_plan(plan)) return rc;
    return mp_set(plan, l_max);
}

int kx_plan_status(kx_plan *plan, int *status_out, kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (!status_out) return set_error(KX_ERR_ARG, "kx_plan_status: NULL output");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int h = 0;
    KX_CUDA_TRY(cudaMemcpyAsync(&h, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    KX_CUDA_TRY(cudaMemsetAsync(plan->d_status, 0, sizeof(int), s));
    KX_CUDA_TRY(cudaStreamSynchronize(s));
    *status_out = h;
    return KX_OK;
}

int kx_selftest_wait(kx_plan *plan, long long max_cycles, kx_stream stream) {
    if (int rc = check_plan(plan)) return rc;
    if (max_cycles < 1 || max_cycles > 2000000000LL) return set_error(KX_ERR_ARG, "kx_selftest_wait: bad limit");
    return selftest_wait(plan, max_cycles, reinterpret_cast<cudaStream_t>(stream));
}

int kx_profile(kx_plan *plan, int enable) {
    if (int rc = check_plan(plan)) return rc;
    plan->prof.on = enable != 0;
    plan->prof.used = 0;
    plan->prof.marks.clear();
    for (int k = 0; k < PK_COUNT; ++k) plan->prof.launches[k] = 0;
    return KX_OK;
}

int kx_profile_read(kx_plan *plan, int n_kinds, double *ms, long long *launches) {
    if (int rc = check_plan(plan)) return rc;
    if (n_kinds < 1 || !ms || !launches) return set_error(KX_ERR_ARG, "kx_profile_read: bad arguments");
    for (int k = 0; k < n_kinds; ++k) {
        ms[k] = 0.0;
        launches[k] = k < PK_COUNT ? plan->prof.launches[k] : 0;
    }
    for (auto &m : plan->prof.marks) {
        cudaEvent_t a = plan->prof.pool[m.second], b = plan->prof.pool[m.second + 1];
        KX_CUDA_TRY(cudaEventSynchronize(b));
        float t = 0.f;
        KX_CUDA_TRY(cudaEventElapsedTime(&t, a, b));
        if (m.first < n_kinds) ms[m.first] += t;
    }
    return KX_OK;
}

int kx_batch_create(int n_sys, kx_plan *const *plans, const int *n_orb, kx_batch **out) {
    if (n_sys < 1 || !plans || !n_orb || !out) return set_error(KX_ERR_ARG, "kx_batch_create: bad arguments");
    *out = nullptr;
    for (int i = 0; i < n_sys; ++i) {
        if (!plans[i]) return set_error(KX_ERR_ARG, "kx_batch_create: NULL plan");
        if (n_orb[i] < 1 || n_orb[i] > 4096) return set_error(KX_ERR_ARG, "kx_batch_create: n_orb out of range");
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i] && n_orb[j] != n_orb[i])
                return set_error(KX_ERR_ARG, "kx_batch_create: a plan shared by two systems needs one n_orb");
    }
    kx_batch *b = new (std::nothrow) kx_batch_s();
    if (!b) return set_error(KX_ERR_NOMEM, "kx_batch_create: host allocation failed");
    b->plans.assign(plans, plans + n_sys);
    b->n_orb.assign(n_orb, n_orb + n_sys);
    // launch shapes: each distinct plan is tuned once at its orbital count
    // (a short budget; shapes tuned earlier in the process are reused), unless
    // KX_AUTOTUNE=0
    const char *at = std::getenv("KX_AUTOTUNE");
    const bool autotune = !(at && std::atoi(at) == 0);
    for (int i = 0; i < n_sys; ++i) {
        bool seen = false;
        for (int j = 0; j < i; ++j) seen = seen || plans[j] == plans[i];
        if (autotune && !seen && !plans[i]->tune.tuned && plans[i]->precision == KX_F16X3) {
            int rc = kx_autotune(plans[i], n_orb[i], 400);
            if (rc) {
                delete b;
                return rc;
            }
        }
    }
    for (int i = 0; i < n_sys; ++i) {
        int rc = reserve(plans[i], n_orb[i]);
        if (rc) {
            delete b;
            return rc;
        }
    }
    cudaGetDevice(&b->device);
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete b;
        return cuda_error(e, "kx_batch_create: stream");
    }
    *out = b;
    return KX_OK;
}

int kx_batch_run(kx_batch *batch, const double *const *psi, double *const *vx_psi, double *e_x, kx_stream stream) {
    if (!batch || !psi || !vx_psi) return set_error(KX_ERR_ARG, "kx_batch_run: bad arguments");
    const int n = (int)batch->plans.size();
    bool same = batch->exec != nullptr && batch->last_ex == e_x;
    for (int i = 0; same && i < n; ++i)
        same = batch->last_psi[i] == psi[i] && batch->last_vx[i] == vx_psi[i] &&
               batch->versions[i] == batch->plans[i]->config_version;
    if (!same) {
        if (batch->exec) cudaGraphExecDestroy(batch->exec);
        if (batch->graph) cudaGraphDestroy(batch->graph);
        batch->exec = nullptr;
        batch->graph = nullptr;
        // the plans may have been used or reconfigured since the last capture:
        // restore each one's full pair list and buffers outside the capture
        for (int i = 0; i < n; ++i)
            if (int rc = reserve(batch->plans[i], batch->n_orb[i])) return rc;
        KX_CUDA_TRY(cudaStreamBeginCapture(batch->cap, cudaStreamCaptureModeThreadLocal));
        int rc = KX_OK;
        for (int i = 0; i < n && rc == KX_OK; ++i)
            rc = dispatch_vx(batch->plans[i], batch->n_orb[i], psi[i], nullptr, vx_psi[i], e_x ? e_x + i : nullptr,
                             false, batch->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(batch->cap, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_error(e, "kx_batch_run: capture");
        batch->graph = g;
        e = cudaGraphInstantiate(&batch->exec, g, 0);
        if (e != cudaSuccess) return cuda_error(e, "kx_batch_run: instantiate");
        batch->last_psi.assign(psi, psi + n);
        batch->last_vx.assign(vx_psi, vx_psi + n);
        batch->last_ex = e_x;
        batch->versions.resize(n);
        for (int i = 0; i < n; ++i) batch->versions[i] = batch->plans[i]->config_version;
    }
    KX_CUDA_TRY(cudaGraphLaunch(batch->exec, reinterpret_cast<cudaStream_t>(stream)));
    return KX_OK;
}

int kx_batch_destroy(kx_batch *batch) {
    if (!batch) return KX_OK;
    if (batch->exec) cudaGraphExecDestroy(batch->exec);
    if (batch->graph) cudaGraphDestroy(batch->graph);
    if (batch->cap) cudaStreamDestroy(batch->cap);
    delete batch;
    return KX_OK;
}

int kx_autotune(kx_plan *plan, int n_orb, int budget_ms) {
    if (int rc = check_plan(plan)) return rc;
    if (n_orb < 1 || n_orb > 4096 || budget_ms < 0) return set_error(KX_ERR_ARG, "kx_autotune: bad arguments");
    if (plan->precision == KX_FP64 || plan->precision == KX_FFT32) return KX_OK;  // single launch shape
    if (tune_lookup(plan, n_orb)) return KX_OK;  // this shape was tuned earlier in the process
    const size_t vec = sizeof(double) * (size_t)n_orb * plan->N;
    double *buf = nullptr;
    KX_CUDA_TRY(cudaMalloc(&buf, 2 * vec + sizeof(double)));
    double *psi = buf, *vx = buf + (size_t)n_orb * plan->N, *ex = vx + (size_t)n_orb * plan->N;
    {
        // deterministic non-trivial orbitals: a smooth bump per orbital
        std::vector<double> h((size_t)n_orb * plan->N);
        for (int k = 0; k < n_orb; ++k)
            for (size_t x = 0; x < plan->N; ++x) {
                size_t x1 = x % plan->n[0], x2 = (x / plan->n[0]) % plan->n[1], x3 = x / (plan->n[0] * plan->n[1]);
                double u = std::sin(3.14159 * (x1 + 1) / (plan->n[0] + 1) * (1 + k % 3)) *
                           std::sin(3.14159 * (x2 + 1) / (plan->n[1] + 1)) *
                           std::sin(3.14159 * (x3 + 1) / (plan->n[2] + 1) * (1 + k % 2));
                h[(size_t)k * plan->N + x] = u;
            }
        cudaMemcpy(psi, h.data(), vec, cudaMemcpyHostToDevice);
    }
    cudaStream_t s;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const TuneParams orig = plan->tune;
    TuneParams best = orig;
    float best_ms = 1e30f;
    const long P = (long)n_orb * (n_orb + 1) / 2;
    // candidates: fused or separate middle passes, pairs per chunk (the default
    // from the workspace budget first, then fixed sizes), A stages of the passes
    const long dflt = [&] {
        TuneParams keep = plan->tune;
        plan->tune.chunk_pairs = 0;
        long c = tc_default_chunk(plan, n_orb);
        plan->tune = keep;
        return c;
    }();
    std::vector<long> chunks = {dflt};
    for (long c : {256L, 512L, 1024L, 2048L})
        if (c != dflt && c <= std::max(2 * P, 256L) && c <= 2 * dflt) chunks.push_back(c);
    const int fuse[] = {1, 0};
    const int stages[] = {0, 2};
    auto t_start = std::chrono::steady_clock::now();
    int rc = KX_OK;
    bool over = false;
    for (int fz : fuse) {
        for (long ch : chunks) {
            for (int st : stages) {
                double elapsed =
                    std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
                if (elapsed > budget_ms && best_ms < 1e30f) {
                    over = true;
                    break;
                }
                plan->tune.fuse_slab = fz;
                plan->tune.chunk_pairs = ch;
                plan->tune.pass_stages = st;
                rc = tc_vx(plan, n_orb, psi, nullptr, vx, ex, false, s);  // warm-up (also sizes the workspace)
                if (rc) break;
                float ms = 1e30f;
                for (int r = 0; r < 3 && rc == KX_OK; ++r) {  // best of three
                    cudaEventRecord(e0, s);
                    rc = tc_vx(plan, n_orb, psi, nullptr, vx, ex, false, s);
                    cudaEventRecord(e1, s);
                    cudaEventSynchronize(e1);
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    ms = std::min(ms, t);
                }
                if (rc) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = plan->tune;
                }
            }
            if (rc || over) break;
        }
        if (rc || over) break;
    }
    if (rc) {
        plan->tune = orig;
    } else {
        plan->tune = best;
        plan->tune.tuned = 1;
        plan->tune.tuned_ms = best_ms;
        tune_store(plan, n_orb);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(buf);
    return rc;
}

int kx_plan_tuning(const kx_plan *plan, long long *chunk_pairs, int *fuse_slab, int *pass_stages, float *tuned_ms) {
    if (int rc = check_plan(plan)) return rc;
    if (chunk_pairs) *chunk_pairs = plan->tune.chunk_pairs;
    if (fuse_slab) *fuse_slab = plan->tune.fuse_slab;
    if (pass_stages) *pass_stages = plan->tune.pass_stages;
    if (tuned_ms) *tuned_ms = plan->tune.tuned ? plan->tune.tuned_ms : 0.f;
    return KX_OK;
}

}  // extern "C"
