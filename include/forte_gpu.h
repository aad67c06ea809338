/*
 * forte_gpu.h -- C ABI of the GB300 CASCI engine: string-driven sigma build,
 * Davidson-Liu eigensolver and spin-free 1-/2-RDMs for a complete active space.
 *
 * The problem statement follows arXiv 2405.10197 (Forte):
 *   - Hamiltonian, Eq. 1 (Sec. II), with the scalar V omitted.  Integrals are
 *     passed in chemist notation (pq|rs) = <pr|qs> (Sec. III "Integral
 *     classes"), so H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs)(E_pq E_rs -
 *     d_qr E_ps) with E_pq = sum_spin a+_p a_q.
 *   - Determinants are alpha string x beta string and the CI vector is the
 *     matrix C[I_alpha][I_beta] (Sec. II.A.1, string-based CI of Handy).
 *   - Strings are n-bit occupation masks (the Determinant class bit layout,
 *     Sec. III), numbered in ascending mask order, so the address of a string
 *     is its colexicographic rank.
 *   - Davidson-Liu diagonalisation (Sec. II.A.1) and the spin-free 1- and
 *     2-RDMs built from the spinful ones of Eqs. (gamma_1), (gamma_2).
 *
 * Conventions for every entry point:
 *   - Return value: FORTE_OK (0) or one of the FORTE_ERR_* codes; the reason
 *     is kept in a thread-local string read by forte_last_error().
 *   - "device" pointers are CUDA global-memory addresses on the context's
 *     device; the caller owns them and they must stay valid until the work
 *     queued on the context's stream has finished.  "host" pointers are plain
 *     CPU memory, read or written before the call returns.
 *   - All vectors are FP64, row-major [nvec][N_alpha][N_beta].
 *   - Work is queued on the context's stream (forte_set_stream; default: the
 *     legacy default stream).  Calls that return host data synchronise it.
 *   - No call traps the GPU; every device-side wait is bounded.
 */
#ifndef FORTE_GPU_H
#define FORTE_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct forte_ctx forte_ctx;
typedef struct forte_sci forte_sci;

enum {
  FORTE_OK = 0,
  FORTE_ERR_ARG = 1,           /* invalid argument (size, pointer, mode) */
  FORTE_ERR_ALLOC = 2,         /* device or host allocation failed */
  FORTE_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  FORTE_ERR_NOT_CONVERGED = 4, /* Davidson hit max_iter; best estimates kept */
  FORTE_ERR_NUMERIC = 5,       /* NaN/Inf in inputs or in residual norms */
  FORTE_ERR_TIMEOUT = 6        /* a bounded device wait gave up */
};

/* Arithmetic of the sigma build (forte_set_precision).  The paper's CASCI
 * (Sec. II.A.1) is FP64 throughout; the reduced-precision modes are an
 * extension: reduced-precision sigma vectors for the bulk of the Davidson
 * iterations, then a refinement with an FP64-class sigma to the requested tolerance. */
enum {
  FORTE_FP64 = 0,   /* every term in FP64 */
  FORTE_TF32 = 1,   /* tensor-core GEMMs (same-spin and alpha-beta) on TF32-rounded
                       operands, FP32 accumulate; Davidson phase on FP32 vectors,
                       then refinement with the FORTE_OZ64 sigma */
  FORTE_BF16X2 = 2, /* as FORTE_TF32 with split hi+lo BF16 operands
                       (hi*hi + hi*lo + lo*hi) */
  FORTE_DF32 = 3,   /* FP64-class sigma in double-FP32 arithmetic: every FP64
                       operand as an unevaluated sum of two FP32 values, exact
                       FP32 products via FMA, compensated sums; relative error
                       ~2^-46 per term.  Davidson as for FORTE_FP64 (FP64 vectors).
                       Not part of the paper's schemes: an FP64 substitute for
                       GPUs whose FP64 pipe is narrow. */
  FORTE_OZ64 = 4    /* FP64-class sigma whose alpha-beta term is formed on the BF16
                       tensor cores from exact products of 8-bit digit slices
                       (integrals and C in 45-bit fixed point per row / 64-string tile,
                       six digits, digit levels up to 8, 64-bit integer sums);
                       same-spin terms as in FORTE_DF32.  Davidson as for
                       FORTE_FP64; also the refinement sigma of FORTE_TF32 /
                       FORTE_BF16X2.  Needs n(n+1)/2 <= 128 (n <= 15) and
                       n_kl(alpha) <= 64; otherwise it is FORTE_DF32.  Not part
                       of the paper's schemes. */
};

/* Build a CAS problem: string lists (a1), signed single-replacement tables
 * (a2), the same-spin string Hamiltonians (a3) and the determinant diagonal
 * H_II (a4).
 *   norb   number of active orbitals n, 1 <= n <= 16
 *   nalpha, nbeta  electron counts, 0 <= n_sigma <= n
 *   h      host [n][n] row-major one-electron integrals, symmetric
 *   eri    host [n][n][n][n] row-major chemist-notation (pq|rs) with the
 *          8-fold permutational symmetry of real orbitals
 * The inputs are copied; the caller keeps ownership.  Returns NULL on error
 * (bad sizes, NULL pointers, NaN/Inf, integrals not symmetric to 1e-12,
 * allocation or CUDA failure); forte_last_error() tells why.  The context
 * uses the current CUDA device at the time of the call.
 * Paper: Eq. 1 (the Hamiltonian) and Sec. II.A.1 (alpha and beta strings, their
 * addressing and single-replacement lists).
 */
forte_ctx *forte_cas_create(int norb, int nalpha, int nbeta, const double *h, const double *eri);

/* Release every device and host resource of the context (NULL is a no-op).
 * Control entry point: the paper has no counterpart.
 */
void forte_destroy(forte_ctx *ctx);

/* Thread-local description of the last error ("" when none).
 * Control entry point: the paper has no counterpart.
 */
const char *forte_last_error(void);

/* Queue subsequent work on this CUDA stream (a cudaStream_t; NULL = legacy
 * default stream).
 * Control entry point: the paper has no counterpart.
 */
int forte_set_stream(forte_ctx *ctx, void *cuda_stream);

/* Select FORTE_FP64, FORTE_TF32, FORTE_BF16X2, FORTE_DF32 or FORTE_OZ64 for forte_sigma,
 * forte_davidson and forte_rdms (every mode but FORTE_FP64 forms the 2-RDM with
 * the tensor-core Gram).  Default FORTE_FP64.  FORTE_ERR_ARG for other values.
 * The paper computes in FP64 (FORTE_FP64); the other modes extend it and have no
 * counterpart there.
 */
int forte_set_precision(forte_ctx *ctx, int mode);

/* N_alpha = C(n, nalpha), N_beta = C(n, nbeta) (host outputs, either may be NULL).
 * Control entry point: the paper has no counterpart.
 */
int forte_get_sizes(const forte_ctx *ctx, long long *n_alpha_str, long long *n_beta_str);

/* Dense single-replacement table of one spin (0 = alpha, 1 = beta), host outputs:
 *   strings [N]        occupation masks, ascending (address = index)
 *   J       [N][n][n]  address of E_pq|I> (a+_p a_q on string I), -1 if it vanishes
 *   sgn     [N][n][n]  its phase (+1/-1), 0 if it vanishes
 * Any output may be NULL.  Phase: (-1)^(occupied orbitals strictly between p and q).
 * Paper: Sec. II.A.1 (string lists and single-replacement lists).
 */
int forte_get_string_tables(const forte_ctx *ctx, int spin, unsigned *strings, int *J,
                            signed char *sgn);

/* Determinant diagonal <I|H|I>, device output [N_alpha][N_beta]; +inf at the
 * determinants an occupation restriction (forte_set_gas) excludes.
 * Paper: Sec. II.A.1 (the diagonal of H, the Davidson-Liu preconditioner).
 */
int forte_get_hdiag(const forte_ctx *ctx, double *hdiag);

/* Occupation-restricted CI (GAS; RAS as its three-space case), Sec. II.A.1:
 * the n active orbitals are split into nspace consecutive spaces of size[g]
 * orbitals (host arrays [nspace]; sizes >= 1 adding up to n), and only the
 * determinants with
 *     gmin[g] <= (alpha + beta electrons in space g) <= gmax[g]   for all g
 * are kept.  Afterwards forte_sigma returns P H P C (P the projector onto the
 * kept determinants: entries of C outside count as zero, those of S are zero),
 * forte_davidson solves P H P in the kept space, and stored guesses are
 * projected.  Vectors keep the full [N_alpha][N_beta] layout, zero outside.
 * The RDM calls act on whatever vectors they are given.  When at most a quarter
 * of the determinants is kept (and the beta strings fall in at most 64
 * occupation classes), sigma has a second exact route besides the full-grid
 * kernels of the precision mode followed by the projection: a kernel over the
 * kept determinants only, in FP64 (FP32 for the FP32 vectors of the
 * reduced-precision Davidson phase), whose cost follows the kept space.  By
 * default the first sigma of each vector type and mode times both routes and
 * keeps the faster (forte_set_gas_route fixes the route).
 * nspace = 0 removes the restriction.  ndet_out (host, may be NULL) receives the number of kept
 * determinants.  FORTE_ERR_ARG for inconsistent sizes or limits, or when no
 * determinant is kept (the previous restriction then stays in force).  Not
 * applied by forte_sigma_fp64_noalloc or forte_batch_solve.  Synchronises the
 * context stream. */
int forte_set_gas(forte_ctx *ctx, int nspace, const int *size, const int *gmin, const int *gmax,
                  long long *ndet_out);

/* Route of the restricted sigma (see forte_set_gas): -1 timed choice (default),
 * 0 full-grid kernels + projection, 1 the kept-determinant kernel (for any
 * restriction with at most 64 beta occupation classes; otherwise the full grid).
 * Clears earlier timings.  FORTE_ERR_ARG for other values.
 * Control entry point: the paper has no counterpart.
 */
int forte_set_gas_route(forte_ctx *ctx, int route);

/* Route the restricted sigma takes for FP64 and FP32 vectors (host outputs, may
 * be NULL): -1 no restriction or not yet timed, 0 full grid, 1 kept
 * determinants; ms (host [4], may be NULL): the timings of the choice, FP64 full
 * grid, FP64 kept, FP32 full grid, FP32 kept (0 when not timed).
 * Control entry point: the paper has no counterpart.
 */
int forte_get_gas_route(const forte_ctx *ctx, int *route_fp64, int *route_fp32, double *ms);

/* Spin-parity sector of the Davidson solve (Sec. II.A.1: projection on states
 * of well-defined total spin), for n_alpha == n_beta (Ms = 0) only.  Exchanging
 * the alpha and beta strings commutes with H, and with alpha creators ordered
 * first a state of total spin S has C[I_beta][I_alpha] = (-1)^S C[I_alpha][I_beta].
 *   parity +1: forte_davidson returns the lowest even-S roots (S = 0, 2, ...)
 *   parity -1: the lowest odd-S roots (S = 1, 3, ...)
 *   parity  0: no restriction (default)
 * Guesses and every new correction vector are projected, x <- (x + parity x^T)/2,
 * so the roots satisfy C^T = parity C exactly.  forte_sigma is not affected.
 * Combines with forte_set_gas.  FORTE_ERR_ARG for other values or n_alpha !=
 * n_beta.  Synchronises the context stream. */
int forte_set_spin_parity(forte_ctx *ctx, int parity);

/* Adaptive configuration interaction (ACI, Sec. II.A.2) on the determinant grid
 * of this CAS, ground state.  Starting from the determinant of lowest H_II as
 * the reference space P, each cycle
 *   - solves H in P (Davidson to `tol`) for Psi_P, E_P;
 *   - forms V = H Psi_P over the whole grid (one FP64-class sigma) and the 2 x 2
 *     estimates eps_mu = D - sqrt(D^2 + V_mu^2), D = (H_mumu - E_P) / 2, for
 *     every determinant outside P;
 *   - excludes the determinants with the smallest |eps| while their summed
 *     |eps| stays at most `sigma` (determinants with equal |eps| leave together);
 *   - solves H in the model space M (every determinant not excluded);
 *   - takes as the next P the determinants of M with the largest c^2 whose
 *     summed c^2 reaches 1 - gamma * sigma (equal values stay together);
 * and stops when P repeats or after max_cycles cycles.  For n_alpha == n_beta
 * the alpha <-> beta mirror determinants have equal estimates and weights in
 * exact arithmetic: both take the larger computed value, and the start P is
 * the lowest determinant with its mirror.  parity (+1 even S, -1 odd S, 0 none;
 * n_alpha == n_beta only) holds the P and M solves to the exchange-parity
 * sector C^T = parity C of the target state; the start determinant is then the
 * lowest one that can carry weight there (I_alpha != I_beta for -1).
 * Outputs: E_out host [2] = {E_M, E_M + sum of the excluded eps}; C_out device
 * [N_alpha][N_beta] or NULL (Psi_M, zero outside M); nM_out, nP_out, cycles_out
 * host or NULL.  The Davidson solves use the context's precision mode; the
 * screening sigma is FP64-class.  The determinant grid is the CAS itself
 * (n <= 16); sigma and the P/M masks cost one grid sweep per Davidson step.
 * FORTE_ERR_ARG for sigma < 0, gamma < 0, max_cycles < 1, tol <= 0, a parity
 * other than -1/0/+1 or with n_alpha != n_beta, or an active forte_set_gas /
 * forte_set_spin_parity.  Synchronises the context stream. */
int forte_aci(forte_ctx *ctx, double sigma, double gamma, int max_cycles, double tol, int parity, double *E_out,
              double *C_out, long long *nM_out, long long *nP_out, int *cycles_out);

/* sigma = H C (Eq. 1 applied in the determinant basis), the hot step a5 + a6.
 *   C  device [nvec][N_alpha][N_beta] FP64 input
 *   S  device [nvec][N_alpha][N_beta] FP64 output, overwritten (not accumulated);
 *      must not overlap C
 *   nvec >= 0 (0 is a no-op)
 * In FORTE_TF32 / FORTE_BF16X2 mode the result carries the reduced precision
 * of that mode.  Asynchronous on the context stream. */
int forte_sigma(forte_ctx *ctx, const double *C, double *S, int nvec);

/* Davidson-Liu solve for the nroots lowest eigenpairs of H in the determinant
 * space (any total spin), to max_k ||H x_k - theta_k x_k||_2 < tol.
 * Guess: unit vectors at the lowest H_II (ties: lowest index), each plus a
 * deterministic perturbation of norm ~0.02 (entries from the splitmix64
 * counter generator) so that closed-shell guesses still reach roots of every
 * spin-flip symmetry sector, orthonormalised; preconditioner
 * (theta - H_II)^-1 with |denominator| clamped to denom_guard; classical
 * Gram-Schmidt, with a second pass when the first removes more than half of
 * the correction's squared norm; subspace collapse (forte_set_davidson_params).
 * When the largest residual has not halved over 50 iterations (the target state
 * is not dominated by the determinants of lowest H_II, where the diagonal
 * preconditioner fails), the solve continues from the Ritz vectors with
 * Jacobi-Davidson (corrections from preconditioned CG on the projected
 * correction equation, thick restart) in the same arithmetic, within the same
 * max_iter budget (Davidson-Liu iterations + Jacobi-Davidson outer steps).
 * In a mixed mode the inner iterations use that mode's sigma and the final
 * residuals and energies are refined with FP64-class sigma builds
 * (Jacobi-Davidson whose inner solves use the mode's sigma) until the FP64
 * residual meets tol.  Results stay in the context (forte_get_roots).
 * Returns FORTE_ERR_NOT_CONVERGED when max_iter is reached (results kept).
 * Paper: Sec. II.A.1 (Davidson-Liu).
 */
int forte_davidson(forte_ctx *ctx, int nroots, double tol);

/* Davidson controls: subspace size and collapse size per root, iteration cap
 * and preconditioner guard.  Defaults 12, 2, 200, 1e-8.
 * Control entry point: the paper has no counterpart.
 */
int forte_set_davidson_params(forte_ctx *ctx, int max_subspace_per_root, int collapse_per_root,
                              int max_iter, double denom_guard);

/* Results of the last forte_davidson: energies (host [nroots], may be NULL),
 * eigenvectors (device [nroots][N_alpha][N_beta], may be NULL; normalised,
 * largest-|c| component positive), final FP64 residual norms (host
 * [nroots], may be NULL) and the iteration count (host, may be NULL).
 * Paper: Sec. II.A.1 (Davidson-Liu results).
 */
int forte_get_roots(const forte_ctx *ctx, double *E, double *C, double *rnorm, int *iters);

/* Restart: use the nvec device vectors [nvec][N_alpha][N_beta] as the initial
 * Davidson subspace of the next forte_davidson call (copied; orthonormalised
 * there).  nvec = 0 restores the unit-vector guess.
 * Paper: Sec. II.A.1 (Davidson-Liu guess vectors).
 */
int forte_set_guess(forte_ctx *ctx, const double *C, int nvec);

/* Spin-free RDMs of one normalised state C (device [N_alpha][N_beta]):
 *   g1 device [n][n]        gamma_pq = sum_s <C|a+_ps a_qs|C>
 *   g2 device [n][n][n][n]  Gamma_pqrs = sum_st <C|a+_ps a+_rt a_st a_qs|C>
 *                           = <E_pq E_rs> - d_qr <E_ps>  (chemist order)
 * Either output may be NULL.  Definitions: Sec. II.A.1, Eqs. (gamma_1),
 * (gamma_2), summed over spin.  FP64. */
int forte_rdms(forte_ctx *ctx, const double *C, double *g1, double *g2);

/* Adjoint of the state-averaged energy E_SA = sum_k w_k E_k (the CI part of the
 * Lagrangian of Sec. II.B, weights w_k of the states) with respect to the
 * integrals.  The E_k are variational, so by Hellmann-Feynman
 *   dE_SA/dh_pq        = sum_k w_k gamma^k_pq
 *   dE_SA/d(pq|rs)     = 1/2 sum_k w_k Gamma^k_pqrs   (each of the n^4 entries of eri
 *                        treated as independent; E = sum h gamma + 1/2 sum (pq|rs) Gamma)
 * and this call ACCUMULATES scale times those into dh (device [n][n]) and
 * deri (device [n]^4).
 *   weights  host [nstates]
 *   C        device [nstates][N_alpha][N_beta], normalised eigenvectors of H
 * FP64.  Asynchronous on the context stream. */
int forte_sa_gradient(forte_ctx *ctx, int nstates, const double *weights, const double *C, double scale,
                      double *dh, double *deri);

/* State-averaged energy E_SA = sum_k w_k E_k (Sec. II.B, the weighted sum over
 * the states of the ensemble) of the first nstates roots of the last
 * forte_davidson on this context.
 *   weights  host [nstates] (any finite values; the paper's ensembles have
 *            w_k >= 0 and sum w_k = 1)
 *   E_sa     host output
 * FORTE_ERR_ARG when nstates < 1 or exceeds the number of roots of the last
 * solve.  Host arithmetic on the stored energies; no device work. */
int forte_sa_energy(const forte_ctx *ctx, int nstates, const double *weights, double *E_sa);

/* One-body transition density matrix between two states (Sec. II.A.1):
 *   t1 device [n][n], t1_pq = sum_s <bra|a+_ps a_qs|ket>.  FP64. */
int forte_tdm1(forte_ctx *ctx, const double *bra, const double *ket, double *t1);

/* Spin-free 3-RDM of one normalised state C (device [N_alpha][N_beta]),
 * Sec. II.A.1, Eq. (gamma_3) summed over spin:
 *   g3 device [n]^6, g3[p][q][r][s][t][u] = sum_{s1 s2 s3}
 *        <C| a+_{p s1} a+_{r s2} a+_{t s3} a_{u s3} a_{s s2} a_{q s1} |C>
 *      = <E_pq E_rs E_tu> - d_qt Gamma_purs - d_st Gamma_pqru
 *        - d_qr (Gamma_pstu + d_st gamma_pu)
 * (chemist order: each pair (p,q), (r,s), (t,u) shares one spin sum).
 * FP64 in every precision mode.  Workspace 2 n^2 N_det doubles plus 64 n^4;
 * work n^2 Gram products of n^2 x n^2 over N_det, so it is meant for the
 * active spaces where the 3-RDM is used (n up to ~10).  Asynchronous on the
 * context stream; FORTE_ERR_ALLOC when the workspace cannot be allocated. */
int forte_rdm3(forte_ctx *ctx, const double *C, double *g3);

/* Batched solve of nprob independent problems (many ActiveSpaceMethod instances
 * of the ActiveSpaceSolver, Sec. III; CASCI of Sec. II.A.1 for each): for problem
 * i, the nroots[i] lowest eigenvalues of its Hamiltonian, written to
 * E_out[offset_i .. offset_i + nroots[i]) with offset_i = sum_{j<i} nroots[j] (host).
 * Inputs per problem as for forte_cas_create (host arrays h[i], eri[i]).
 * Problems with equal (norb, nalpha, nbeta) form a size class sharing strings,
 * replacement lists and the same-spin sparsity pattern.  A class runs either as
 * ONE kernel launch with one CTA per problem that runs the whole Davidson-Liu
 * solve on the device (the class launches are captured in one CUDA graph and use
 * one pooled device allocation), or on the single-problem path (forte_cas_create /
 * forte_davidson with the tensor-core sigma of the chosen mode) on 8 worker
 * threads with their own streams, concurrently with the class launches.  Before
 * the solve an autotuner times, for every class, the per-CTA sigma for each
 * (threads per CTA, beta tile width) candidate and keeps the fastest; it then
 * times one Davidson iteration of the class's first problem on the
 * single-problem path and sends the class there when
 *   P x t_single_iteration < t_CTA_sigma x ceil(P / (resident CTAs per SM x SMs)).
 * Problems with more than 100,000 determinants or more than 3 roots always take
 * the single-problem path.  forte_batch_tuning reports the choices.
 *   precision  FORTE_FP64: FP64 sigma; FORTE_DF32 / FORTE_OZ64: double-FP32
 *              (FP64-class) sigma; FORTE_TF32 / FORTE_BF16X2: FP32 sigma down to
 *              a residual of max(tol, 3e-4), then the double-FP32 sigma (class
 *              launches; the single-problem path uses that mode's own solver).
 *              Vectors, subspace and eigenproblem are FP64 in every mode.
 *   tol        max residual 2-norm per root; max_iter the iteration cap (<= 0: 400)
 * Davidson as forte_davidson (guess, preconditioner, 12 vectors per root,
 * collapse to 2 per root); a problem whose in-CTA solve does not converge within
 * max_iter is solved again on the single-problem path (which continues a stalled
 * Davidson-Liu with Jacobi-Davidson).  status_out (host [nprob], may be NULL) gets each
 * problem's status.  Returns the worst status (FORTE_ERR_NOT_CONVERGED keeps
 * energies); FORTE_ERR_ALLOC when the pooled workspace (about
 * (2 * 12 * nroots + 2 * nroots + 4) * N_det doubles per class-launch problem)
 * cannot be allocated.  Synchronous. */
int forte_batch_solve(int nprob, const int *norb, const int *nalpha, const int *nbeta, const int *nroots,
                      const double *const *h, const double *const *eri, int precision, double tol,
                      int max_iter, double *E_out, int *status_out);

/* Autotuner choices of the last forte_batch_solve, one entry per size class below
 * the in-CTA limits (host outputs of length max_classes, any may be NULL;
 * *nclass = number of classes): orbital and electron counts, threads per CTA,
 * beta tile width of the alpha-beta term, the measured time (ms) of one sigma
 * build of the class's first problems (one CTA each) with the chosen candidate,
 * the chosen path (0: class launch, 1: single-problem path), the measured time
 * (ms) of one single-problem-path Davidson iteration, the class's problem count
 * and the resident CTAs per SM of its launch.
 * Control entry point: the paper has no counterpart.
 */
int forte_batch_tuning(int max_classes, int *nclass, int *norb, int *nalpha, int *nbeta, int *threads, int *tile,
                       double *sigma_ms, int *path, double *single_iter_ms, int *problems, int *ctas_per_sm);

/* Problem counts of the last forte_batch_solve (host outputs, may be NULL): solved
 * in class launches, sent to the single-problem path, and solved again on the
 * single-problem path after their in-CTA Davidson-Liu did not converge.
 * Control entry point: the paper has no counterpart.
 */
int forte_batch_stats(int *class_launch, int *single_path, int *retried);

/* FP64 sigma = H C that allocates no device memory (the paper has no
 * counterpart; this is a service for callers of the library).  It is meant for
 * callers that cannot call cudaMalloc during the call: code whose device memory
 * belongs to another allocator (a framework's caching allocator, a fixed memory
 * budget) and latency-critical loops where cudaMalloc/cudaFree, which may
 * synchronise the device, are not acceptable.  forte_sigma grows scratch
 * buffers on demand; this entry point instead uses a fixed 16 MB array built
 * into the library, which every GPU that loads the library holds until exit.
 *   C, S, nvec  as for forte_sigma (device pointers, FP64, S overwritten,
 *               S must not overlap C); always FP64 whatever forte_set_precision says
 * Limit: nvec * N_alpha * N_beta <= 1,048,576 (e.g. one CAS(12,12) vector);
 * larger requests return FORTE_ERR_ARG without touching the GPU.
 * The first call on a device looks up the array's device address (with that
 * device made current) and keeps it for the process; make that first call
 * before any stream capture.  The address belongs to the device's primary
 * context: do not call this entry point again after cudaDeviceReset.  All
 * calls share the array, so calls that overlap on the GPU (for instance on two
 * streams at once) race.  Same kernels as forte_sigma in FP64 (traced like them
 * under forte_profile_enable).  Asynchronous on the context stream. */
int forte_sigma_fp64_noalloc(forte_ctx *ctx, const double *C, double *S, int nvec);

/* Status of the bounded device waits (no counterpart in the paper: failure
 * reporting of this library).  The tensor-core kernels (alpha-beta, same-spin,
 * digit-slice sigma and 2-RDM Gram) bound every pipeline wait by a clock budget;
 * when one expires the CTA raises the context's device status flag, the other
 * roles stop, the CTA waits (with the fixed default budget) for its own MMAs and
 * copies in flight, frees its tensor memory and exits -- it never traps the GPU.
 * forte_get_status synchronises the context stream and returns FORTE_ERR_TIMEOUT
 * (and clears the flag) when such a wait expired since the last check, else
 * FORTE_OK; forte_davidson and forte_rdms check it themselves.  The outputs of the
 * affected call are undefined; the context stays usable. */
int forte_get_status(forte_ctx *ctx);

/* Clock budget (cycles) of one pipeline wait of the context's tensor-core kernels;
 * 0 restores the default (4e9 cycles, about two seconds).  Meant for tests of the
 * failure path: a budget of a few cycles makes the waits expire.  Synchronises the
 * context stream.
 * Control entry point: the paper has no counterpart.
 */
int forte_set_wait_budget(forte_ctx *ctx, unsigned long long cycles);

/* Kernel tracing.  While enabled, every kernel this library launches for the
 * context is bracketed by CUDA events on the context stream (on = 1 also
 * clears earlier records; on = 0 stops recording and keeps them).
 * Control entry point: the paper has no counterpart.
 */
int forte_profile_enable(forte_ctx *ctx, int on);

/* Launch count and summed device time (ms) of the recorded launches whose
 * kernel name equals `kernel` (NULL: all kernels).  Synchronises the stream.
 * Host outputs; either may be NULL.
 * Control entry point: the paper has no counterpart.
 */
int forte_profile_query(forte_ctx *ctx, const char *kernel, int *launches, double *total_ms);

/* Name of the i-th distinct recorded kernel (NULL when i is out of range);
 * the string lives as long as the library.
 * Control entry point: the paper has no counterpart.
 */
const char *forte_profile_kernel_name(forte_ctx *ctx, int i);

/* Number of vectors pushed through the sigma build since the context was
 * created, in FP64 and in a reduced-precision mode (host outputs, may be NULL).
 * Control entry point: the paper has no counterpart.
 */
int forte_get_counters(const forte_ctx *ctx, long long *sigma_vectors_fp64,
                       long long *sigma_vectors_mixed);

/* ---- determinant-list sigma (selected CI, Sec. II.A.2) ----
 *
 * Handle holding the integrals of an n-orbital problem for sigma over arbitrary
 * lists of determinants, the data path of adaptive CI: no string tables, so n may
 * exceed the CAS grid's limit.  norb in 1..32; h [norb][norb], eri
 * [norb]^4 (chemist order) host arrays, copied to the current device.  Returns
 * NULL (reason in forte_last_error) for a bad norb, NULL or non-finite integrals,
 * or a failed device allocation.  Release with forte_sci_destroy. */
forte_sci *forte_sci_create(int norb, const double *h, const double *eri);
/* Frees the list context and its device memory (NULL is accepted).
 * Control entry point: the paper has no counterpart.
 */
void forte_sci_destroy(forte_sci *sci);
/* Stream of the handle's work (default: the legacy default stream).
 * Control entry point: the paper has no counterpart.
 */
int forte_sci_set_stream(forte_sci *sci, void *cuda_stream);

/* S[v][i] = sum_j <D_i|H|D_j> C[v][j] over a list of determinants (H of Eq. 1;
 * the elements follow the Slater-Condon rules, pairs more than two replacements
 * apart vanish).
 *   dets  device [ndet] 64-bit words: alpha orbital p at bit p, beta orbital p at
 *         bit norb + p (creation operators ordered by that index, alpha first);
 *         any order, any mix of (n_alpha, n_beta) sectors (sectors do not couple);
 *         a word listed twice counts twice
 *   C, S  device [nvec][ndet] FP64; S overwritten, must not overlap C
 *   ndet >= 0 (<= 2^31), nvec >= 0; 0 is a no-op
 * Every pair (i, j) is screened by popcount(D_i ^ D_j) <= 4 (cost ndet^2 / 32
 * warp steps), so the call suits lists up to ~1e6 determinants.  Deterministic:
 * per-row sums are taken in list order within fixed splits, added in split order.
 * Asynchronous on the handle's stream; grows a scratch buffer (nvec <= 4 at a time
 * x splits x ndet doubles) on demand. */
int forte_sci_sigma(forte_sci *sci, long long ndet, const uint64_t *dets, const double *C, double *S, int nvec);

#ifdef __cplusplus
}
#endif
#endif /* FORTE_GPU_H */
