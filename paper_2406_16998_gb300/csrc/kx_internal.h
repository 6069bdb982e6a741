// Internal declarations shared by the kronx translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/kronx.h"

namespace kx {

// Thread-local error state behind kx_last_error_detail().
int set_error(int code, const std::string &msg);
int cuda_error(cudaError_t e, const char *what);

#define KX_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return ::kx::cuda_error(_e, #expr); \
    } while (0)

#define KX_LAUNCH_CHECK(what)                               \
    do {                                                    \
        cudaError_t _e = cudaGetLastError();                \
        if (_e != cudaSuccess) return ::kx::cuda_error(_e, what); \
    } while (0)

constexpr int kMaxN = 128;       // per-axis limit of the library
constexpr int kOrbBlock = 4;     // orbitals per block of the pair enumeration
constexpr int kGroupSlots = 2 * kOrbBlock;

// One accumulation group: the pairs of one orbital block pair (I, J), I <= J
// (a contiguous run of items), touching at most kGroupSlots orbitals.
struct Group {
    int first_item;
    int n_items;
    int n_slots;
    int orb[kGroupSlots];
};
constexpr int kTile = 128;       // tcgen05 M (rows of pencils per tile)
constexpr float kVScale = 16384.f;  // V operand scale 2^14 (|V| <= 1)
constexpr int kVScaleExp = 14;

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Launch-shape choices kept per plan (set by kx_autotune).
struct TuneParams {
    long chunk_pairs = 0;     // pairs per chunk (0 = choose from the workspace budget)
    int fuse_slab = 1;        // fuse the mode-2/mode-1 products of each k3 slice into one kernel
    int pass_stages = 0;      // shared A stages of the pass kernels (0 = as many as fit, at most 4)
    int tuned = 0;            // set by kx_autotune (or taken from the process-wide table of tuned shapes)
    float tuned_ms = 0.f;     // best apply time measured by the tuner
};

// Per-launch CUDA-event timing by kernel kind (kx_profile / kx_profile_read).
enum ProfKind { PK_PREP = 0, PK_X3F, PK_X2F, PK_X1, PK_X2I, PK_X3I, PK_FINAL, PK_FP64_MODE, PK_FP64_OTHER,
                PK_ACE, PK_SETUP, PK_ACC, PK_SLAB, PK_ACE_COMB, PK_MP, PK_FFT, PK_BLOCH, PK_BLOCH_OTHER, PK_COUNT };
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;       // reusable events
    size_t used = 0;
    std::vector<std::pair<int, size_t>> marks;  // (kind, index of the start event; stop = +1)
    long long launches[PK_COUNT] = {0};
};

// Device workspace, grown on demand and reused across calls.
struct Workspace {
    void *ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace kx

namespace kx {
// Called by the split path when rows [o0, o1) of the caller's Vx psi output are
// final (written on stream s).
struct FinalHook {
    void (*fn)(void *ctx, int o0, int o1, cudaStream_t s) = nullptr;
    void *ctx = nullptr;
};
// Orbitals that arrive in pieces (kx_vx_apply_host): piece k holds orbitals
// [end[k-1], end[k]) and is on the device once ready[k] has completed; the
// split path waits for (and converts) a piece only before the first chunk that
// needs it.
struct InputPieces {
    std::vector<int> end;
    std::vector<cudaEvent_t> ready;
};
}  // namespace kx

struct kx_plan_s {
    int n[3];
    double h[3];
    int bc[3];
    int fd_order;
    int kind;
    double omega;
    int precision;
    int device;
    int num_sms;
    size_t N;
    double dV;
    double fmax = 0.0;  // max of the f table (set-up)
    int np[3];  // per-axis size padded to a multiple of 16 (tensor-core K and N)

    // float64 set-up (device)
    double *d_lam[3] = {nullptr, nullptr, nullptr};   // n[a]
    double *d_V[3] = {nullptr, nullptr, nullptr};     // n[a] x n[a], row-major V[x][k]
    double *d_f64 = nullptr;                          // N, index k1 + n1 (k2 + n2 k3)
    float *d_f32 = nullptr;                           // N, same layout

    // tensor-core operands (device): per axis, hi and lo fp16 blocks of the
    // np x np zero-padded, 2^14-scaled V in 8x8 core-matrix order
    __half *d_Vs[3] = {nullptr, nullptr, nullptr};    // [2][np*np]: hi block then lo block
    // KX_FFT32 plans: twiddles exp(-2 pi i t / n_a) (3 x 128 complex) and f in DFT order (N)
    float *d_fft_tw = nullptr;
    float *d_fft_f = nullptr;

    int *d_status = nullptr;                          // bounded-wait status word

    kx::TuneParams tune;
    kx::Workspace ws;        // chunk buffers and per-pair scratch
    kx::Workspace ws_host;   // device staging for kx_vx_apply_host
    // Pair enumeration (orbital blocks of kx::kOrbBlock, see ensure_pairs) and its
    // accumulation groups, rebuilt when n_orb or the pair range changes.
    int ws_norb = -1;
    long long pr_begin = -1, pr_end = -1;
    // explicit block-pair list (kx_vx_apply_block_pairs): when blk_mode is set,
    // ensure_pairs enumerates the block pairs of blk_req instead of a range;
    // blk_cur is the list the current enumeration was built from (empty: range)
    bool blk_mode = false;
    std::vector<int> blk_req, blk_cur;
    int *d_pairs = nullptr;       // int2 per item (i, j), i <= j
    int *d_item_slot = nullptr;   // int2 per item: slots of i and j inside its group
    int *d_groups = nullptr;      // kx::Group per group
    size_t pairs_cap = 0, groups_cap = 0;
    std::vector<int> h_group_first;  // first item of each group (+ sentinel)
    std::vector<int> h_orb_last;     // per orbital: index of the last group that touches it (-1: none)
    kx::Profiler prof;
    // kx_vx_apply_host: told when leading rows of Vx psi are final, so that their
    // device-to-host copies run on copy_stream while later chunks compute
    kx::FinalHook final_hook;
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> copy_events;
    kx::InputPieces in_pieces;                // set only for the duration of a host-buffer call
    cudaStream_t h2d_stream = nullptr;
    std::vector<cudaEvent_t> h2d_events;
    std::vector<int> h_group_maxorb;          // per group: its largest orbital index
    // pair {i, j} in the current pair range (n_orb x n_orb bytes, symmetric)
    unsigned char *d_pair_mask = nullptr;
    size_t pair_mask_cap = 0;
    // multipole boundary values (kx_plan_set_multipole): order, number of
    // harmonics K = (l_max + 1)^2, and per harmonic the regular solid harmonic
    // R_k and the correction field h_k on the grid (K x N, float64 and float32)
    int mp_lmax = -1;
    int mp_K = 0;
    double *d_mpR = nullptr, *d_mpH = nullptr;
    float *d_mpR32 = nullptr, *d_mpH32 = nullptr;
    float *d_mpMax = nullptr;  // max |R_k| (K values) then max |h_k| (K values)
    bool mp_applied = false;   // the split path applied the correction inside its pair loop
    bool mp_grad = false;      // kx_energy_gradient: use the symmetric form of the correction
    // bumped whenever device buffers a captured batch graph refers to are
    // reallocated or refilled (workspaces, pair list, multipole fields)
    unsigned long long config_version = 0;
    kx::Workspace mp_scratch;
};

namespace kx {

// Bracket one kernel launch with profiling events (no-ops unless kx_profile is on).
int prof_begin(kx_plan *p, int kind, cudaStream_t s);
int prof_end(kx_plan *p, cudaStream_t s);

// ---- set-up (kx_setup.cu)
int plan_setup(kx_plan *p);          // eig, f tables, split operands (synchronous)
void plan_free(kx_plan *p);

// ---- workspace (kx_capi.cu)
int ensure_workspace(kx_plan *p, size_t bytes);
int ensure_pairs(kx_plan *p, int n_orb, cudaStream_t s, long long begin = 0, long long end = -1);

// ---- FP64 path (kx_fp64.cu)
int fp64_apply_fL(kx_plan *p, int n_rhs, const double *b, double *x, cudaStream_t s);
int fp64_vx(kx_plan *p, int n_orb, const double *psi, const double *occ, double *vx, double *ex,
            bool energy_only, cudaStream_t s, long pair_begin = 0, long pair_end = -1);
size_t fp64_workspace_bytes(const kx_plan *p, long chunk);

// ---- tensor-core path (kx_tc.cu)
int tc_apply_fL(kx_plan *p, int n_rhs, const double *b, double *x, cudaStream_t s);
int tc_vx(kx_plan *p, int n_orb, const double *psi, const double *occ, double *vx, double *ex,
          bool energy_only, cudaStream_t s, long pair_begin = 0, long pair_end = -1);
size_t tc_workspace_bytes(const kx_plan *p, int n_orb, long chunk);
long tc_default_chunk(const kx_plan *p, int n_orb);
int selftest_wait(kx_plan *p, long long max_cycles, cudaStream_t s);
int tc_apply_fL_noalloc(kx_plan *p, int n_rhs, const double *b, double *x, cudaStream_t s);

// ---- ACE tail (kx_ace.cu)
int ace_run(kx_plan *p, int n_orb, const double *psi, const double *W, double *xi, double *M_out,
            cudaStream_t s);
int ace_apply_run(kx_plan *p, int n_xi, const double *xi, int n_vec, const double *phi, double *out,
                  cudaStream_t s);
// ---- fully periodic grids through the DFT (kx_fft.cu)
bool fft_supported(const int *n, const int *bc);
int fft_setup(kx_plan *p);
size_t fft_partial_count(const kx_plan *p, long chunk);
// f(L) of R items: sources psi_i psi_j (pairs) or src32 (rhs), complex scratch C
// (R x N), output real part into out32 (fp32) or out64; energy into ex
int fft_passes(kx_plan *p, long R, const int2 *pairs, const float *src32, int rhs, const double *occ, float2 *C,
               float *out32, double *out64, double *ex, double *partial, bool energy_only, cudaStream_t s);

// ---- Bloch-periodic boundary conditions and k-point sums (kx_bloch.cu)
// Vx of n_vec complex vectors phi at k-point k (out overwritten); psi is
// n_kpt x n_orb x N complex (interleaved float64), occ n_kpt x n_orb (nullable),
// theta (n_kpt x 3) and wk (n_kpt) host arrays.
int bloch_vx_apply(kx_plan *p, int n_kpt, const double *theta, const double *wk, int n_orb, const double *psi,
                   const double *occ, int k, int n_vec, const double *phi, double *out, cudaStream_t s);
// Vx psi_nk for every k-point (vx like psi) and, if ex, E_x into ex[0], from the
// k-point blocks [b_begin, b_end) of the (k, q >= k) enumeration (all of them:
// [0, n_kpt (n_kpt + 1) / 2)).
int bloch_vx_all(kx_plan *p, int n_kpt, const double *theta, const double *wk, int n_orb, const double *psi,
                 const double *occ, long long b_begin, long long b_end, double *vx, double *ex, cudaStream_t s);
// E_x alone into ex[0] (forward transforms and Parseval).
int bloch_energy(kx_plan *p, int n_kpt, const double *theta, const double *wk, int n_orb, const double *psi,
                 const double *occ, double *ex, cudaStream_t s);

// ---- multipole boundary values (kx_mp.cu)
int mp_set(kx_plan *p, int l_max);
void mp_free(kx_plan *p);
int mp_reserve(kx_plan *p, int n_orb);
int mp_reserve_scratch(kx_plan *p, int n_orb);
// tensor-core form of the Vx psi correction: written into the float32
// accumulator of the split path before its pair loop (sets mp_applied)
bool mp_tc_eligible(const kx_plan *p, int n_orb, const double *psi);
int mp_correct_into_acc(kx_plan *p, int n_orb, const double *psi, const double *occ, float *acc, double *ex,
                        cudaStream_t s);
// Vx psi and E_x (or E_x alone) of the pair range of the last ensure_pairs:
// adds the rank-K boundary correction to the homogeneous result
int mp_correct_vx(kx_plan *p, int n_orb, const double *psi, const double *occ, double *vx, double *ex,
                  bool energy_only, cudaStream_t s);
// x += sum_k Q_k(b) h_k for n_rhs right-hand sides b
int mp_correct_apply(kx_plan *p, int n_rhs, const double *b, double *x, cudaStream_t s);

// out[a][b] = scale sum_x A_a(x) B_b(x) w(x) over the grid (w nullable; the
// float64 weights serve float64 plans, the float32 ones the others), partial
// sums per grid-point range added in float64 in a fixed order.  Uses the plan
// workspace (grid_projection_bytes).
size_t grid_projection_bytes(const kx_plan *p, int na, int nb);
int grid_projection(kx_plan *p, const double *A, int na, const double *B, int nb, const double *w64, const float *w32,
                    double scale, double *out, cudaStream_t s, int kind = PK_ACE);
// out = (accumulate ? out : 0) + sgn A C for na grid vectors A and the na x nb
// row-major float64 matrix C; no workspace.
int grid_combination(kx_plan *p, const double *A, int na, const double *C, int nb, double sgn, bool accumulate,
                     double *out, cudaStream_t s, int kind = PK_ACE_COMB);

}  // namespace kx
