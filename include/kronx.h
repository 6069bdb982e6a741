/*
 * kronx — exact-exchange operator on a finite-difference grid through the
 * Kronecker-product representation of f(L), for one GPU (sm_103a).
 *
 * Method: Jing & Suryanarayana, "Efficient real space formalism for hybrid
 * density functionals" (arXiv 2406.16998).
 *
 *   Sec. 2, Eqs. 3-5:  (Vx psi)_i = -sum_j g_j psi_j * phi_ij,
 *                      phi_ij     = f(L) (psi_i * psi_j),
 *                      E_x        = -1/2 dV sum_ij g_i g_j <psi_i psi_j, phi_ij>.
 *   Sec. 3, Eqs. 11-19: L = I3(x)I2(x)L1 + I3(x)L2(x)I1 + L3(x)I2(x)I1,
 *                      Lk = Vk Lambda_k Vk^T,
 *                      f(L) b = (V3(x)V2(x)V1) f(l1+l2+l3) (V3(x)V2(x)V1)^T b,
 *                      applied as three mode products, a diagonal scaling and
 *                      three inverse mode products (Roth's relationship, Eq. 19).
 *   Kernel f (Sec. 3 after Eq. 18): unscreened f = -4 pi / lambda; screened
 *                      f = (4 pi / mu)(1 - exp(-mu / (4 w^2))), mu = -lambda,
 *                      f(0) = pi / w^2 (the transform of erfc(w r)/r, Sec. 2.2).
 *
 * Conventions shared by every call
 *   - Grid vectors have N = n1*n2*n3 entries, x1 fastest, then x2, then x3.
 *   - Orbital blocks are n_orb grid vectors stored one after the other
 *     (orbital k occupies elements [k*N, (k+1)*N)), float64.
 *   - Unless a call says "host", every pointer argument is a device pointer on
 *     the current CUDA device, owned by the caller, and must stay valid until
 *     the work queued on `stream` has finished.  Plans, batches and their
 *     workspaces are owned by the library.
 *   - Work is queued asynchronously on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream).  Calls return before the GPU has finished.
 *   - Every call returns 0 (KX_OK) or a KX_ERR_* code; no C++ exception crosses
 *     this boundary.  kx_last_error_detail() gives a one-line explanation of the
 *     last failure on the calling host thread.
 *   - Integration weights: <a, b> = dV * sum(a * b), dV = h1*h2*h3.
 *   - A plan owns one workspace: calls on the same plan must be issued from one
 *     host thread and on one stream at a time (or be ordered by the caller);
 *     different plans are independent.  Complex grid vectors (k-point calls)
 *     are interleaved (re, im) float64 pairs, 16-byte aligned.
 */
#ifndef KRONX_H
#define KRONX_H

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque handles. */
typedef struct kx_plan_s kx_plan;
typedef struct kx_batch_s kx_batch;
/* cudaStream_t-compatible stream handle. */
typedef struct CUstream_st *kx_stream;

/* Boundary condition per axis (Sec. 2: Dirichlet in vacuum directions,
 * periodic in extended directions). */
#define KX_DIRICHLET 0
#define KX_PERIODIC  1

/* Kernel f (Sec. 3, after Eq. 18). */
#define KX_UNSCREENED 0 /* f = -4 pi / lambda            (PBE0, Eq. 5)  */
#define KX_SCREENED   1 /* erfc(w r)/r, w = kx_kernel.omega (HSE, Eq. 10) */

/* Arithmetic of the mode products. */
#define KX_FP64  0 /* plain float64 on the CUDA cores (the baseline path)            */
#define KX_F16X3 1 /* tensor cores: fp16 hi/lo split of both operands, three products
                      (hi*hi + hi*lo + lo*hi) accumulated in fp32, per-pair power-of-two
                      scaling; energy and outputs accumulated in fp32/fp64.
                      BF16X3, BF16X6 and TF32X3 splits were considered and dropped on
                      purpose: an fp16 hi + lo pair carries 22 significand bits at the
                      bf16 rate with three products, where bf16 x3 carries 16 bits
                      (short of the 1e-5 / 1e-6 targets), bf16 x6 needs twice the
                      products and tf32 runs at half the fp16 rate with twice the
                      operand bytes; fp16's narrow exponent range is handled by
                      the power-of-two scales                                        */
#define KX_FFT32 2 /* fully periodic grids only: f(L) through the DFT (the eigenvectors of
                      a periodic axis are Fourier modes), float32 complex Stockham FFTs
                      of radix 2, 3, 4, 5 (axes of 80 points: a 16 x 5 four-step
                      transform in registers); every n[a] a product of 2, 3 and 5,
                      at most 128 (KX_ERR_UNSUPPORTED otherwise); the FFT variant the
                      Kronecker form is compared with (Sec. 3, Fig. 1)                */

/* Error codes. */
#define KX_OK              0
#define KX_ERR_ARG         1 /* invalid argument (sizes, pointers, enum values)        */
#define KX_ERR_SINGULAR    2 /* unscreened kernel with all axes periodic: lambda = 0   */
#define KX_ERR_NOMEM       3 /* a device or host allocation failed                    */
#define KX_ERR_CUDA        4 /* a CUDA runtime call or kernel launch failed            */
#define KX_ERR_TIMEOUT     5 /* a bounded wait inside a kernel ran out                 */
#define KX_ERR_UNSUPPORTED 6 /* valid request outside what the library implements     */

/* Grid and finite-difference operator (Sec. 3, Eqs. 11-12).
 *   n[a]      points per axis, 2 <= n[a] <= 128; for KX_F16X3, n[a] % 8 == 0.
 *   h[a]      spacing (bohr), > 0.
 *   bc[a]     KX_DIRICHLET (homogeneous, unknowns at x_i = (i+1) h) or
 *             KX_PERIODIC (x_i = i h, circulant Lk).
 *   fd_order  even, 2..24: centred stencil of half-width fd_order/2. */
typedef struct {
    int n[3];
    double h[3];
    int bc[3];
    int fd_order;
} kx_grid;

/* Kernel choice: kind = KX_UNSCREENED or KX_SCREENED, omega (bohr^-1) > 0 for
 * the screened kernel. */
typedef struct {
    int kind;
    double omega;
} kx_kernel;

/* kx_plan_create — set-up of one grid/kernel (Sec. 3, Eqs. 12-13 and the f
 * table of Eq. 19).  Builds L1, L2, L3, diagonalises each on the GPU in float64
 * (cyclic Jacobi), evaluates f(l1_i + l2_j + l3_k) for all N spectral points in
 * float64, and prepares the operands of the chosen precision.  Synchronous:
 * returns after the set-up kernels have finished.
 *   grid, kernel   host pointers, read only during the call.
 *   precision      KX_FP64 or KX_F16X3.
 *   out            host pointer receiving the plan handle.
 * Errors: KX_ERR_ARG, KX_ERR_SINGULAR (unscreened and every axis periodic),
 * KX_ERR_UNSUPPORTED (sizes outside the limits above), KX_ERR_NOMEM, KX_ERR_CUDA. */
int kx_plan_create(const kx_grid *grid, const kx_kernel *kernel, int precision, kx_plan **out);

/* kx_plan_destroy — frees the plan and its workspaces (synchronises the device
 * first).  NULL is accepted. */
int kx_plan_destroy(kx_plan *plan);

/* kx_plan_eig — copies the float64 set-up of one axis to host memory:
 * lam[n] (eigenvalues of L_axis, ascending) and V[n*n] (row-major, V[x*n + k] is
 * component x of eigenvector k), so that L_axis V = V diag(lam) (Sec. 3, Eq. 13).
 * Either host pointer may be NULL.  Synchronous. */
int kx_plan_eig(const kx_plan *plan, int axis, double *lam, double *V);

/* kx_plan_ftable — copies the float64 f table (N entries, index
 * k1 + n1*(k2 + n2*k3), value f(l1_k1 + l2_k2 + l3_k3)) to host memory.
 * Synchronous. */
int kx_plan_ftable(const kx_plan *plan, double *f);

/* kx_energy_gradient — dE_x/dpsi_a(x) of the discrete E_x (Sec. 2, Eq. 5 as a
 * dV-weighted sum over the pairs) for the orbitals psi, and E_x:
 *   grad_a = 2 dV g_a G_a,
 * G = Vx psi for zero boundary values (the solve is symmetric in rho); with
 * multipole boundary values (kx_plan_set_multipole) the solve
 * K rho = f(L) rho + sum_k Q_k(rho) h_k is not symmetric and
 *   G_a = (Vx psi with zero boundary values)_a
 *         - 1/2 sum_j g_j psi_j sum_k (Q_k(rho_aj) h_k + P_k(rho_aj) R_k),
 * P_k(rho) = dV <h_k, rho>, the gradient of E_x = -1/2 dV sum g_i g_j
 * <rho_ij, K rho_ij> (the symmetric part (K + K^T) / 2 enters).
 *   psi   in: n_orb grid vectors (device);  occ: nullable (device)
 *   grad  out: n_orb grid vectors (device), must not overlap psi
 *   e_x   out (nullable): E_x (device scalar)
 * Same precision and arguments as kx_vx_apply. */
int kx_energy_gradient(kx_plan *plan, int n_orb, const double *psi, const double *occ, double *grad, double *e_x,
                       kx_stream stream);

/* kx_plan_set_multipole — Dirichlet boundary values from the multipole
 * expansion of the source (Sec. 4: for isolated systems the boundary values of
 * each linear system come from the multipole expansion of the Coulomb kernel
 * and enter through the right-hand side) for every later solve of this plan:
 *   phi = f(L) (rho + L_ext phi_ext / (4 pi)),
 * phi_ext = the expansion of rho's potential to order l_max about the box
 * centre ((n_a + 1) h_a / 2 per axis), taken at the exterior points the FD
 * stencil reaches across each face.  Solved as f(L) rho plus a rank-K
 * correction sum_k Q_k(rho) h_k, K = (l_max + 1)^2, with the fields h_k set up
 * here by K float64 solves.  Applies to kx_apply_fL, kx_vx_apply,
 * kx_vx_apply_pairs, kx_vx_apply_host (which then copies Vx psi back after the
 * last chunk), kx_energy and batches created afterwards.
 *   l_max  0..8; -1 turns the expansion off (zero boundary values again).
 * KX_ERR_UNSUPPORTED unless all three axes are Dirichlet and the kernel is
 * unscreened; while it is on, kx_apply_fL_noalloc returns KX_ERR_UNSUPPORTED
 * and tensor-core plans accept at most 256 orbitals.  Synchronous; allocates
 * 24 K N bytes of fields. */
int kx_plan_set_multipole(kx_plan *plan, int l_max);

/* kx_apply_fL — X = f(L) B for n_rhs independent right-hand sides (Sec. 3,
 * Eq. 18-19).  b and x hold n_rhs grid vectors each (float64); b is read only,
 * x must not overlap b.  n_rhs >= 0 (0 is a no-op). */
int kx_apply_fL(kx_plan *plan, int n_rhs, const double *b, double *x, kx_stream stream);

/* kx_apply_fL_noalloc — kx_apply_fL for callers that cannot allocate device
 * memory at the point of the call (no counterpart in the paper).  Such callers
 * reserved their device memory up front (a pool or caching allocator owns it,
 * or a solver loop must not pay the device-wide synchronisation of cudaMalloc
 * and cudaFree between iterations).  This entry point allocates nothing: its
 * scratch is a static device array of 30 MiB + 160 KiB inside the library,
 * which every GPU that loads the library's tensor-core module holds until the
 * process exits.  The plan (created earlier with kx_plan_create, KX_F16X3
 * precision) and the caller's b and x are the only other memory it touches.
 *   Limit: n_rhs * N <= 2,621,440 grid values per call; larger requests return
 *   KX_ERR_ARG with the numbers (split them into several calls).
 *   Every call looks up the array's device address (cudaGetSymbolAddress, which
 *   allocates nothing) with the plan's device current, so no address is kept
 *   across a cudaDeviceReset.  The first call on a device may load the
 *   library's tensor-core device code and the array with it, as any first
 *   launch does; make that first call before any stream capture.
 *   All calls share the array and it keeps the previous call's contents (the
 *   entry point clears what must start at zero); calls whose GPU work overlaps
 *   (different streams or host threads on one device) race on it.
 * Arguments as in kx_apply_fL; the current device must be the plan's. */
int kx_apply_fL_noalloc(kx_plan *plan, int n_rhs, const double *b, double *x, kx_stream stream);

/* kx_vx_apply — the exact-exchange apply and energy (Sec. 2, Eqs. 3-5 / 8-10 at
 * the Gamma point, one spin channel).  Every unordered pair (i <= j) is solved
 * once (n_orb (n_orb+1)/2 solves of Eq. 19).
 *   psi     n_orb orbitals (float64), read only.
 *   occ     n_orb occupations g (float64) or NULL for g = 1.
 *   vx_psi  out: n_orb grid vectors (float64), (Vx psi)_i; must not overlap psi.
 *   e_x     out: one float64, E_x = -1/2 dV sum_ij g_i g_j <rho_ij, phi_ij>;
 *           may be NULL.
 * n_orb >= 1. */
int kx_vx_apply(kx_plan *plan, int n_orb, const double *psi, const double *occ,
                double *vx_psi, double *e_x, kx_stream stream);

/* kx_vx_apply_pairs — the part of kx_vx_apply contributed by a contiguous range
 * [pair_begin, pair_end) of the library's list of the n_orb (n_orb+1)/2
 * unordered pairs (i <= j).  The list groups orbitals in blocks of four
 * (block b = orbitals 4b .. 4b+3 of nb blocks, the last possibly shorter) and
 * visits the block pairs (I, J), I <= J, in this order: those of the leading
 * block columns J < jc column-major (J = 0 .. jc-1, I = 0 .. J), jc being the
 * fewest columns that hold ceil(15% of nb (nb+1)/2) block pairs, then the rest
 * row-major (I = 0 .. nb-1, J = max(I, jc) .. nb-1); inside a diagonal block
 * (I, I) the pairs i <= j row-major, inside an off-diagonal block all (i, j)
 * row-major.
 * vx_psi and e_x receive the
 * partial sums of Eqs. 3-5 over that range (overwritten, not added), so that
 * ranges covering the list sum to the full result: the unit a multi-GPU split
 * of the pair solves (Sec. 3: the O(Nk^2 Ns^2) systems are independent)
 * reduces.  0 <= pair_begin <= pair_end <= n_orb (n_orb+1)/2; other arguments
 * as in kx_vx_apply. */
int kx_vx_apply_pairs(kx_plan *plan, int n_orb, const double *psi, const double *occ,
                      long long pair_begin, long long pair_end, double *vx_psi, double *e_x,
                      kx_stream stream);

/* kx_vx_apply_block_pairs — the part of kx_vx_apply contributed by an explicit
 * set of orbital block pairs: the unit of a two-dimensional block-cyclic split
 * of the pair solves across GPUs (Sec. 3: the pair systems are independent;
 * the paper's own split is by bands and domains, Sec. 4).  Orbitals are
 * grouped in blocks of four as in kx_vx_apply_pairs; block pair (I, J), I <= J,
 * holds the pairs (i, j) with i in block I and j in block J (i <= j when I = J).
 *   blocks    HOST array of 2 * n_blocks ints, (I, J) per block pair, 0 <= I
 *             <= J < ceil(n_orb / 4), each block pair at most once, any order;
 *             read during the call only.
 *   n_blocks  0 .. nb (nb + 1) / 2 (0 gives zeros).
 *   vx_psi, e_x receive the partial sums of Eqs. 3-5 over those pairs
 *   (overwritten): block-pair sets that partition the list sum to kx_vx_apply.
 * Other arguments as in kx_vx_apply. */
int kx_vx_apply_block_pairs(kx_plan *plan, int n_orb, const double *psi, const double *occ,
                            const int *blocks, int n_blocks, double *vx_psi, double *e_x,
                            kx_stream stream);

/* kx_vx_apply_host — kx_vx_apply on HOST buffers (pinned memory recommended):
 * copies psi (and occ) to library-owned device buffers, runs the apply and
 * copies vx_psi and e_x back; returns after all of it has finished.  With
 * KX_F16X3 the rows of vx_psi whose pairs are all done are copied back on a
 * plan-owned stream while the remaining pairs compute (the work starts on
 * `stream` and ends joined to it).  psi, occ (nullable), vx_psi, e_x
 * (nullable) are host pointers.  Calls on one plan must not overlap. */
int kx_vx_apply_host(kx_plan *plan, int n_orb, const double *psi, const double *occ,
                     double *vx_psi, double *e_x, kx_stream stream);

/* kx_energy — E_x alone (no inverse transforms): by Parseval, with V orthogonal,
 * <rho, f(L) rho> = sum_k f(Lambda)_k ((V^T rho)_k)^2 (Sec. 3, Eq. 15-16).
 * Arguments as in kx_vx_apply; e_x must not be NULL. */
int kx_energy(kx_plan *plan, int n_orb, const double *psi, const double *occ, double *e_x,
              kx_stream stream);

/* kx_ace — adaptively compressed exchange tail (the ACE construction that
 * Sec. 4 cites; float64 throughout):
 *   M = dV psi^T W (n_orb x n_orb, W = vx_psi),  -M = R^T R (Cholesky, R upper),
 *   xi = W R^{-1}, so that -xi (dV xi^T psi) = W.
 *   psi, vx_psi  inputs (n_orb grid vectors each).
 *   xi           out: n_orb grid vectors; must not overlap the inputs.
 *   M_out        out (nullable): n_orb*n_orb float64, row-major, M before factoring.
 * M, its Cholesky factor and R^{-1} are float64; the grid-sized products
 * (Psi^T W and W R^{-1}) are float64 for KX_FP64 plans and float32 products
 * with float64 sums across blocks of grid points for KX_F16X3 plans.
 * Returns KX_ERR_ARG if -M is not positive definite (detected on the GPU; the
 * call then synchronises the stream to read the flag).  1 <= n_orb <= 256. */
int kx_ace(kx_plan *plan, int n_orb, const double *psi, const double *vx_psi, double *xi,
           double *M_out, kx_stream stream);

/* kx_ace_apply — the compressed exchange operator built by kx_ace applied to
 * vectors (the ACE construction Sec. 4 cites):
 *   out = -xi (dV xi^T phi),
 * which equals Vx phi for phi in the span of the orbitals xi was built from,
 * so an SCF loop can use it in place of Vx between rebuilds.
 *   xi    in: n_xi grid vectors (device), as written by kx_ace.
 *   phi   in: n_vec grid vectors (device).
 *   out   out: n_vec grid vectors (device); must not overlap xi or phi.
 * The projections dV xi^T phi (n_xi x n_vec) are summed in float64.  The
 * grid-sized products run in float64 for KX_FP64 plans and as float32
 * products with float64 sums across blocks of grid points for KX_F16X3
 * plans (relative error ~1e-7 of the largest entry).  Queued on the stream,
 * no host synchronisation.  1 <= n_xi <= 256, n_vec >= 1; KX_ERR_ARG
 * otherwise. */
int kx_ace_apply(kx_plan *plan, int n_xi, const double *xi, int n_vec, const double *phi, double *out,
                 kx_stream stream);

/* Bloch-periodic boundary conditions and k-point sums (Sec. 2.1, Eqs. 6-9;
 * Sec. 3, Eq. 19 with complex, wavevector-dependent Vk), one spin channel (the
 * spin sum adds independent channels).  The plan's KX_PERIODIC axes become
 * Bloch-periodic; its Dirichlet axes (vacuum) ignore the k-point phases.
 *   n_kpt  number of k-points (1..1024).
 *   theta  host, n_kpt x 3: phase per cell of each k-point along each axis,
 *          theta_a = k_a n_a h_a (radians); entries of Dirichlet axes unused.
 *          The pair (mq, nk) is solved with the Bloch phases theta_k - theta_q.
 *   wk     host, n_kpt Brillouin-zone weights w_q.
 *   n_orb  bands per k-point (1..4096).
 *   psi    in: n_kpt x n_orb x N complex grid values, interleaved (re, im)
 *          float64 (device, 16-byte aligned), psi[q][m][x].
 *   occ    in: n_kpt x n_orb occupations g_mq (device) or NULL for 1.
 * The forward transform contracts each axis with conj(Vk), the inverse with Vk;
 * along a Bloch axis Vk[x][m] = e^{i (2 pi m + theta) x / n} / sqrt(n).  The mode
 * products run in complex float64 on the CUDA cores for KX_FP64 plans; for the
 * others in complex float32 data, on the tensor cores (fp16 hi/lo split
 * products, fp32 accumulation) along axes of 32 or 64 points and on the CUDA
 * cores along the rest, with float64 accumulation of Vx across bands (relative
 * error ~1e-6).  The environment variable KX_BLOCH_TC, read at each call, is a
 * bit mask of the axes allowed the tensor-core products (default all; 0 none).
 * A bounded wait inside a tensor-core product that runs out records
 * KX_ERR_TIMEOUT in the plan status (kx_plan_status).  Queued on the stream,
 * no host synchronisation.
 * KX_ERR_UNSUPPORTED for plans with multipole boundary values; KX_ERR_SINGULAR
 * does not arise past kx_plan_create (an unscreened plan has a Dirichlet axis
 * or is rejected there). */

/* kx_vx_apply_kpoint — Vx applied to n_vec complex vectors phi (device,
 * n_vec x N, layout of psi) at k-point k_index:
 *   out_v = -sum_q w_q sum_m g_mq psi_mq f(L_{k-q}) (conj(psi_mq) phi_v).
 * out (device, n_vec x N complex) must not overlap psi or phi.  KX_ERR_ARG for
 * sizes out of range, NULL or misaligned buffers. */
int kx_vx_apply_kpoint(kx_plan *plan, int n_kpt, const double *theta, const double *wk, int n_orb,
                       const double *psi, const double *occ, int k_index, int n_vec, const double *phi,
                       double *out, kx_stream stream);

/* kx_vx_kpoints — Vx psi_nk at every k-point into vx (device, layout of psi,
 * not overlapping it) and, if ex != NULL, the exchange energy
 *   E_x = 1/2 dV sum_k w_k sum_n g_nk Re <psi_nk, Vx psi_nk>
 * (Eq. 8 after the Poisson solves) into ex[0] (device float64).  The pairs
 * of k-points k < q are solved once for both: the solve of (q m, k n) is the
 * complex conjugate of that of (k n, q m), so n_kpt (n_kpt + 1) / 2 blocks of
 * n_orb^2 solves are done. */
int kx_vx_kpoints(kx_plan *plan, int n_kpt, const double *theta, const double *wk, int n_orb, const double *psi,
                  const double *occ, double *vx, double *ex, kx_stream stream);

/* kx_vx_kpoint_blocks — the part of kx_vx_kpoints that the k-point blocks
 * [block_begin, block_end) contribute, for a split across GPUs: the blocks are
 * (k, q), q >= k, numbered k-major (k = 0: q = 0..n_kpt-1, then k = 1: q =
 * 1..n_kpt-1, ...; n_kpt (n_kpt + 1) / 2 of them); block (k, q) adds q's bands
 * to Vx psi_k and, for q > k, k's bands to Vx psi_q.  vx (layout of psi) is
 * overwritten with the partial sums of every k-point and ex[0] (if not NULL)
 * with the matching partial E_x, so that the partials of disjoint ranges
 * covering all blocks add up to kx_vx_kpoints.  Other arguments as
 * kx_vx_kpoints; KX_ERR_ARG for a range outside [0, n_kpt (n_kpt + 1) / 2]. */
int kx_vx_kpoint_blocks(kx_plan *plan, int n_kpt, const double *theta, const double *wk, int n_orb,
                        const double *psi, const double *occ, long long block_begin, long long block_end, double *vx,
                        double *ex, kx_stream stream);

/* kx_energy_kpoints — E_x alone (Eq. 8) into ex[0] (device float64, required)
 * through Parseval: -1/2 dV sum w_k w_q g_nk g_mq sum f(Lambda) |V^H rho|^2,
 * rho = conj(psi_mq) psi_nk; only the forward transforms of the blocks
 * (k, q), q >= k, are computed (the block (q, k) has the conjugate
 * coefficients and counts twice).  Arguments as kx_vx_kpoints. */
int kx_energy_kpoints(kx_plan *plan, int n_kpt, const double *theta, const double *wk, int n_orb,
                      const double *psi, const double *occ, double *ex, kx_stream stream);

/* kx_batch_create — groups n_sys plans (different grids, kernels and orbital
 * counts) into one CUDA graph that runs every system's kx_vx_apply.  Each
 * distinct KX_F16X3 plan that is not tuned yet is first passed to kx_autotune
 * at its orbital count with a 400 ms budget (shapes tuned earlier in the
 * process are reused; KX_AUTOTUNE=0 in the environment skips this).
 * Workspaces are reserved here so that the graph holds no allocation.
 *   plans[n_sys], n_orb[n_sys]  host arrays.  out: host pointer for the handle. */
int kx_batch_create(int n_sys, kx_plan *const *plans, const int *n_orb, kx_batch **out);

/* kx_batch_run — replays the graph on `stream`.  psi[s], vx_psi[s] (host arrays
 * of device pointers) are system s's orbitals and output; e_x (device, n_sys
 * float64, nullable) receives each system's E_x.  The graph is re-captured when
 * the pointer set differs from the previous run. */
int kx_batch_run(kx_batch *batch, const double *const *psi, double *const *vx_psi, double *e_x,
                 kx_stream stream);

/* kx_batch_destroy — frees the batch (not its plans).  NULL is accepted. */
int kx_batch_destroy(kx_batch *batch);

/* kx_autotune — times the launch shapes the library offers for `plan` at n_orb
 * orbitals and keeps the fastest in the plan: fused or separate middle passes
 * (the k3-slice kernel or three pass kernels), pairs per chunk (the default
 * from the workspace budget and fixed sizes 256 .. 2048), and the number of
 * shared-memory A stages of the pass kernels.  Each candidate is timed as the
 * best of three applies after a warm-up, on an internal stream, with synthetic
 * orbitals (smooth products of sines: the timing does not depend on the
 * values), until budget_ms milliseconds have passed.  The choice is also kept
 * in a process-wide table keyed by grid, precision, device model and n_orb:
 * a later call for the same shape takes it from there without timing.
 * KX_FP64 and KX_FFT32 plans have a single launch shape (no-op).  Synchronous;
 * allocates 16 n_orb N bytes for the duration of the call. */
int kx_autotune(kx_plan *plan, int n_orb, int budget_ms);

/* kx_plan_tuning — the plan's current launch-shape choices (host pointers,
 * each may be NULL): pairs per chunk (0 = from the workspace budget), fused
 * middle passes (1) or not (0), pass-kernel A stages (0 = as many as fit), and
 * the best apply time the tuner measured (0 if the plan was not tuned). */
int kx_plan_tuning(const kx_plan *plan, long long *chunk_pairs, int *fuse_slab, int *pass_stages,
                   float *tuned_ms);

/* kx_plan_status — reads and clears the plan's device status word (set by a
 * kernel whose bounded wait ran out).  Synchronises `stream`.  *status_out
 * receives KX_OK or KX_ERR_TIMEOUT.  status_out is a host pointer. */
int kx_plan_status(kx_plan *plan, int *status_out, kx_stream stream);

/* kx_selftest_wait — failure-path self-test of the bounded waits the kernels
 * use (no counterpart in the paper): one CTA waits on an mbarrier phase that
 * nothing completes, gives up after max_cycles SM clock cycles
 * (1 <= max_cycles <= 2e9), records KX_ERR_TIMEOUT in the plan's status word
 * and returns; read the word with kx_plan_status.  The GPU context stays usable. */
int kx_selftest_wait(kx_plan *plan, long long max_cycles, kx_stream stream);

/* kx_profile — starts (enable = 1, clearing earlier records) or stops (0)
 * per-launch CUDA-event timing of the plan's kernels on the stream each is
 * launched on.  Launch counts are kept whether or not timing is on. */
int kx_profile(kx_plan *plan, int enable);

/* kx_profile_read — per kernel kind k < n_kinds: total event-timed
 * milliseconds ms[k] and launch count launches[k] since the last kx_profile
 * call (host arrays).  Kinds: 0 prep (fp64 -> fp32), 1 X3F (rho = psi_i psi_j,
 * mode 3 forward), 2 X2F (mode 2 forward), 3 X1 (mode 1 forward, f(Lambda)
 * scaling and energy, mode 1 inverse), 4 X2I (mode 2 inverse), 5 X3I (mode 3
 * inverse and Vx psi accumulation), 6 finalize/energy sums, 7 float64 mode
 * products, 8 other float64 kernels, 9 ACE projections, 10 set-up, 11 accumulation of
 * g psi phi into Vx psi, 12 fused mode 2 forward + X1 + mode 2 inverse per
 * k3 slice (replaces kinds 2-4 where the operands fit in shared memory),
 * 13 ACE combinations of grid vectors (xi = W R^{-1}, -xi P); kind 9 covers
 * the ACE projections over the grid and their reduction; 14 the multipole
 * boundary correction (moments of the sources, correction of the solution,
 * Vx psi and E_x), 15 the DFT passes of KX_FFT32 plans, 16 the complex mode
 * products of the Bloch k-point path, 17 its other kernels (bases, f tables,
 * conversions, Vx accumulation, E_x sums).
 * Synchronises on the recorded events. */
int kx_profile_read(kx_plan *plan, int n_kinds, double *ms, long long *launches);

/* kx_last_error_detail — copies the last error message of the calling host
 * thread into buf (host, len bytes, NUL-terminated).  Returns the last code. */
int kx_last_error_detail(char *buf, int len);

/* kx_strerror — static name of an error code. */
const char *kx_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* KRONX_H */
