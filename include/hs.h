/*
 * hs.h - C ABI of the GB300 nested shift-invert MINRES library for the
 * periodic spin-1/2 random-field Heisenberg chain (Kutsuzawa & Todo,
 * arXiv:2203.09732).
 *
 *   H = sum_{j=1..L} ( S_j . S_{j+1} - h_j Sz_j ),  S_{L+1} = S_1,  J = 1
 *                                                       (Sec. I, Eq. (1))
 * in the Sz = 0 sector of even L (dimension n = C(L, L/2)).
 *
 * Conventions shared by every call:
 *   - Basis: site j (1-based) is bit j-1 of a 32-bit word, bit = 1 is spin up.
 *     The sector states are ranked in ascending integer order; vectors are
 *     n contiguous elements in that order, on the device unless the argument
 *     name ends in _host.
 *   - Ownership: the caller owns every vector argument; the handle owns its
 *     tables, workspace and CUDA graphs and frees them in hs_free.
 *   - Streams: all work is enqueued on the stream given to hs_create (NULL =
 *     legacy default stream). Calls that return host results synchronise that
 *     stream before returning.
 *   - Memory: a handle's device memory comes from a memory pool the library
 *     owns, allocated and freed in order on the handle's stream, so creating
 *     and freeing handles does not synchronise the device while solves run on
 *     other streams. Freed memory stays in the pool for later handles until
 *     the process exits; pinned host staging buffers are likewise reused.
 *   - Concurrency: handles on separate streams run concurrently. With more
 *     than 8 busy streams, set CUDA_DEVICE_MAX_CONNECTIONS (up to 32) in the
 *     environment before the process creates its CUDA context; otherwise
 *     streams share hardware queues and a short kernel can wait behind
 *     another stream's persistent solve.
 *   - Errors: every call returns an hs_status; no call aborts, throws or traps.
 *     hs_last_error() returns a message for the last failing call on a handle.
 *     Device-side failures (non-finite values, breakdown) are reported through
 *     the status, never by a device trap.
 */
#ifndef HS_H
#define HS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hs_handle hs_handle;

typedef enum {
  HS_OK = 0,
  HS_BAD_ARG = 1,        /* invalid size, pointer, L, h, sigma or option       */
  HS_OOM = 2,            /* device or host allocation failed                    */
  HS_CUDA = 3,           /* a CUDA runtime call failed                          */
  HS_NOT_CONVERGED = 4,  /* iteration cap reached before the tolerance          */
  HS_BREAKDOWN = 5,      /* gamma_k = 0 in MINRES, or a Lanczos breakdown       */
  HS_NONFINITE = 6,      /* NaN/Inf met in a reduction                          */
  HS_TIMEOUT = 7         /* reserved: bounded device wait expired               */
} hs_status;

typedef enum { HS_F32 = 0, HS_F64 = 1 } hs_dtype;

/* Diagonal preconditioners M of Sec. II: identity; Jacobi diag|a_ii - sigma|;
 * row norm r_i = sqrt(|a_ii - sigma|^2 + sum_{k != i} |a_ik|^2). */
typedef enum { HS_PC_ID = 0, HS_PC_JACOBI = 1, HS_PC_ROWNORM = 2 } hs_precond;

typedef struct {
  long long iters;     /* total MINRES iterations (all refinement sweeps)        */
  int sweeps;          /* FP64 refinement sweeps (1 for plain FP64 MINRES)        */
  int status;          /* hs_status of the solve                                  */
  double phi;          /* last |phi_k| / beta_1 of the last inner solve           */
  double resid_minv;   /* final ||b - (H - sigma) x||_{M^-1} / ||b||_{M^-1}, FP64 */
  double resid_2;      /* final ||b - (H - sigma) x||_2 / ||b||_2, FP64          */
  int form;            /* solver form of the (last inner) solve: HS_FORM_*        */
  int pad;
} hs_minres_info;

/* Solver forms (all run the recurrence of Algorithm 2): vectors resident in
 * shared memory (chains up to L = 20 in FP64, 22 in FP32); superblock passes
 * (from L = 24 on); one persistent cooperative kernel with vectors in global
 * memory; per-pass kernels replayed from a CUDA graph; and the shared-memory
 * form with one global reduction per iteration (the product taken of
 * M^-1 p_k, p carried by the recurrence of q and replaced by a product every
 * R steps, beta_{k+1}^2 expanded in sums known before alpha_k: equal in exact
 * arithmetic, different in rounding). */
enum { HS_FORM_SMEM = 1, HS_FORM_SUPERBLOCK = 2, HS_FORM_PERSISTENT = 3, HS_FORM_GRAPH = 4,
       HS_FORM_SMEM1 = 5 };

typedef struct {
  int steps;           /* Lanczos steps taken (k at exit)                         */
  int converged;       /* number of wanted pairs meeting the tolerance           */
  long long minres_iters; /* MINRES iterations summed over all solves            */
  int sweeps;          /* refinement sweeps summed over all solves               */
  double sigma;        /* shift used                                              */
  double max_resid;    /* max_i ||H psi_i - E_i psi_i||_2 (FP64, certified)       */
  double seconds_solve;   /* host wall time inside the MINRES solves             */
  double seconds_total;   /* host wall time of the whole call                    */
  double seconds_ritz;    /* host wall time of the Ritz extraction and the FP64  */
                          /* certification of the K pairs (part of the total)    */
  int unconverged_solves; /* MINRES solves that stopped at their iteration cap   */
                          /* before minres_tol; the step still used them         */
  int pad;
} hs_lanczos_info;

/* Create a handle for chain length L (even, 4 <= L <= 32) and fields
 * h_host[0..L-1] (h_host[j-1] = h_j of Eq. (1); finite). sigma is the shift of
 * Algorithm 1; pass NaN to set sigma = (E_min + E_max) / 2 (Sec. IV A), found
 * by an extremal FP64 Lanczos run on the device. cuda_stream is a
 * cudaStream_t (may be NULL). Builds the ranking tables on the host and
 * copies them to the current device. On failure *out is NULL. */
hs_status hs_create(int L, const double* h_host, double sigma, void* cuda_stream,
                    hs_handle** out);

/* Free the handle and everything it owns (synchronises its stream first). */
void hs_free(hs_handle* hd);

/* Message for the last failed call on hd ("" if none; static text if hd NULL). */
const char* hs_last_error(const hs_handle* hd);

/* n = C(L, L/2). */
hs_status hs_dim(const hs_handle* hd, long long* n_out);

/* Current sigma; hs_set_sigma replaces it (finite). Cached solver graphs stay
 * valid: sigma is read from device memory at run time. */
hs_status hs_get_sigma(const hs_handle* hd, double* sigma_out);
hs_status hs_set_sigma(hs_handle* hd, double sigma);

/* Extremal eigenvalues by plain FP64 Lanczos on H (three-term recurrence,
 * T_k re-diagonalised every 10 steps) until both move by < tol; returns
 * E_min, E_max and (E_min + E_max) / 2 without changing the handle's sigma.
 * Sec. IV A defines sigma from these. */
hs_status hs_extremal(hs_handle* hd, int max_steps, double tol, double* emin_out,
                      double* emax_out, double* mid_out);

/* Ranking of the Sz = 0 sector (row a1): states_dev[t] = the state of rank
 * first + t, t < count (bit-exact, ascending integer order). */
hs_status hs_unrank(hs_handle* hd, long long first, long long count,
                    unsigned int* states_dev);
/* ranks_dev[t] = rank of states_dev[t], or -1 if the word is not an L-bit word
 * of popcount L/2. */
hs_status hs_rank(hs_handle* hd, const unsigned int* states_dev, long long count,
                  long long* ranks_dev);

/* diag_dev[i] = a_ii (diagonal of H, FP64, may be NULL); minv_dev[i] = 1 / M_ii
 * of preconditioner pc at the current sigma (FP64, may be NULL). Sec. II. */
hs_status hs_diag(hs_handle* hd, double* diag_dev, hs_precond pc, double* minv_dev);

/* Matrix-free y = H x (shifted = 0) or y = (H - sigma) x (shifted = 1), in
 * FP32 (x, y float, FP32 accumulation) or FP64. x and y must not overlap and
 * must be aligned to their element size (any offset from that is fine).
 * Eq. (1); element (i, k) for i != k is 1/2 exactly when states i and k differ
 * by the flip of one antiparallel bond (Appendix C). From L = 24 on, FP32 uses
 * the superblock form (x of two superblocks staged in shared memory); the
 * environment variable HS_HV_SB=0 selects the block form, HS_HV_SB=1 the
 * superblock form for both precisions from L = 22 on. Both forms give the
 * same values up to the order of the row sums. */
hs_status hs_matvec(hs_handle* hd, const void* x_dev, void* y_dev, hs_dtype dtype,
                    int shifted);

/* Solve (H - sigma) x = b by the preconditioned MINRES of Algorithm 2
 * (Appendix A), x0 = 0, stopping when |phi_k| <= tol * beta_1 or after kmax
 * iterations (kmax <= 0: 20 n).
 *   mixed = 0: plain FP64 MINRES.
 *   mixed = 1: FP32 MINRES (FP32 vectors and H x, FP64 scalar recurrences)
 *              inside FP64 iterative refinement of the residual
 *              r = b - (H - sigma) x, until ||r||_{M^-1} <= tol ||b||_{M^-1}
 *              (each sweep runs to the relative tolerance inner_tol; <= 0: 1e-5).
 * b_dev and x_dev are FP64, n elements, may not overlap. info may be NULL.
 * Returns HS_NOT_CONVERGED (x still holds the last iterate) if the cap is hit. */
hs_status hs_minres(hs_handle* hd, const double* b_dev, double* x_dev, double tol,
                    long long kmax, hs_precond pc, int mixed, double inner_tol,
                    hs_minres_info* info);

/* One FP32 MINRES solve without refinement (Algorithm 2 in FP32 vectors,
 * FP64 scalars): b_dev, x_dev float. For tests of the FP32 inner solver. */
hs_status hs_minres_f32(hs_handle* hd, const float* b_dev, float* x_dev, double tol,
                        long long kmax, hs_precond pc, hs_minres_info* info);

/* The K eigenpairs of H nearest sigma by the nested shift-invert Lanczos of
 * Algorithm 1 with full reorthogonalisation (two classical Gram-Schmidt
 * passes) and MINRES inside every step.
 *   K >= 1; m_max: Lanczos step cap (<= 0: max(130, 3K + 30)); tol: stop when
 *   every wanted Ritz pair has beta_{k+1} |y_{k,i}| <= tol |theta_i|;
 *   seed: SplitMix64 stream of the start vector (entries uniform on [-1, 1));
 *   v0_dev: optional FP64 start vector (overrides seed); mixed, pc, inner_tol:
 *   as hs_minres, with MINRES tolerance minres_tol; minres_kmax: iteration cap
 *   of each MINRES solve, all refinement sweeps together (<= 0: 50 n). A solve
 *   that reaches the cap still feeds its iterate into the step and is counted
 *   in info->unconverged_solves (a capped run measures the cost of every part
 *   of the pipeline on problems whose full solve takes too long).
 * Outputs: evals_host[K] ordered by |E - sigma| (ties by E), E_i the Rayleigh
 * quotient of psi_i; evecs_dev (K x n FP64, vector i at evecs_dev + i n; may be
 * NULL); resid_host[K] = ||H psi_i - E_i psi_i||_2 (may be NULL).
 * Workspace: m_max + 8 FP64 vectors plus the MINRES vectors. */
hs_status hs_lanczos_eigs(hs_handle* hd, int K, int m_max, double tol,
                          unsigned long long seed, const double* v0_dev, int mixed,
                          hs_precond pc, double minres_tol, double inner_tol,
                          long long minres_kmax, double* evals_host, double* evecs_dev,
                          double* resid_host, hs_lanczos_info* info);

/* End-to-end convenience call with host buffers only: creates a handle on the
 * current device (its own stream; persistent solves limited to sm_budget SMs,
 * 0 = all), runs hs_lanczos_eigs, computes the twist overlaps (z_host, 2K
 * doubles, may be NULL), copies the eigenvectors to evecs_host (K x n, may be
 * NULL) and frees everything. sigma NaN = midpoint. */
hs_status hs_eigs_host(int L, const double* h_host, double sigma, int K, int m_max,
                       double tol, unsigned long long seed, int mixed, hs_precond pc,
                       double minres_tol, double inner_tol, long long minres_kmax,
                       int sm_budget, double* evals_host, double* evecs_host,
                       double* resid_host, double* z_host, hs_lanczos_info* info);

/* Batched disorder sweep (Sec. IV B-C: |z|^2 averaged within each realisation,
 * then across realisations). B realisations, L_host[r] (even, 4..32, at most
 * two distinct values) and fields h_host (the realisations' L_host[r] values
 * concatenated in order), each with sigma = (E_min + E_max) / 2 and the start
 * vector of seed + r. One persistent cooperative launch runs them all: CTA
 * groups take realisations from one queue per chain length and run all of
 * Algorithm 1 on each on the device (FP64 inner solves by Algorithm 2 with pc,
 * relative tolerance minres_tol, at most 50 n iterations; full
 * reorthogonalisation; the convergence test on T_k); m (m_max, else
 * max(130, 3K + 30)) is at most 256. The group size per (L, pc, SM count) is
 * timed on first use and cached in the JSON file HS_SWEEP_TUNE (default
 * $HOME/.cache/hs_sweep_tune.json); HS_SWEEP_S forces it.
 * Outputs (host, realisation r at offset r K): evals_host (B K, each ordered as
 * by hs_lanczos_eigs and certified the same way), resid_host (B K FP64
 * residuals ||H psi - E psi||, may be NULL), z_host (2 B K: Re, Im of the twist
 * overlaps, may be NULL), zz_host (B: the mean of |z|^2 over the realisation's
 * K pairs, may be NULL).
 * HS_NOT_CONVERGED (outputs written) when some realisation's pairs did not
 * converge; other errors leave the outputs undefined. Uses the current device;
 * allocates its own stream, handles and workspace and frees them. */
typedef struct {
  int realisations;      /* B                                                      */
  int converged;         /* realisations whose K pairs all converged               */
  int max_steps;         /* Lanczos steps of the longest realisation               */
  int launches;          /* solver launches of the sweep (1)                       */
  int nclass;            /* distinct chain lengths (1 or 2)                        */
  int pad;
  long long minres_iters;
  int L[2];              /* per chain length: L,                                   */
  int S[2];              /*   CTAs per group,                                      */
  int groups[2];         /*   groups,                                              */
  int tuned[2];          /*   1 timed now, 0 from the cache, -1 forced             */
  double zz_mean[2];     /*   mean over realisations of the per-realisation mean   */
  double zz_std[2];      /*   of |z|^2, and its sample standard deviation          */
  double max_resid;      /* largest FP64 residual of all pairs                     */
  double seconds_setup;  /* handles, sigma, start vectors, schedule                */
  double seconds_solve;  /* the launch                                             */
  double seconds_total;
} hs_sweep_info;

hs_status hs_sweep(int B, const int* L_host, const double* h_host, int K, int m_max, double tol,
                   unsigned long long seed, double minres_tol, hs_precond pc,
                   double* evals_host, double* resid_host, double* z_host, double* zz_host,
                   hs_sweep_info* info);

/* Twist overlap z_i = <psi_i| U_twist |psi_i>, U_twist = exp[i 2pi/L sum_j j Sz_j]
 * (Sec. III), for K real FP64 vectors psi_dev + i n (not normalised by the
 * call). z_host[2 i] = Re z_i, z_host[2 i + 1] = Im z_i. */
hs_status hs_twist(hs_handle* hd, const double* psi_dev, int K, double* z_host);

/* Twist overlaps without any device allocation, for callers that cannot call
 * cudaMalloc (code inside someone else's stream capture, plug-ins whose host
 * application owns every device allocation, processes that already hold
 * nearly all device memory). The paper has no counterpart; it computes the
 * same z_i as hs_twist, with no handle.
 *   L: even, 4 <= L <= 32; psi_dev: K FP64 vectors of n = C(L, L/2) entries in
 *   rank order (vector i at psi_dev + i n); 1 <= K <= 8 (the fixed scratch holds
 *   8 vectors; larger K returns HS_BAD_ARG); z_dev: 2K doubles on the device,
 *   z_dev[2i] = Re z_i, z_dev[2i+1] = Im z_i; cuda_stream: where the work is
 *   enqueued (asynchronous, nothing is synchronised).
 * Scratch: a fixed 512 KiB static device array inside this library (held by
 * every GPU that loads it until the process exits); no cudaMalloc, cudaFree
 * or allocating library routine is called. Each call made outside a stream
 * capture looks up the array's device address (cudaGetSymbolAddress) with the
 * current device; a call inside a capture reuses the address found by the last
 * uncaptured call on that device, so make one call on each device before any
 * stream capture (and again after a cudaDeviceReset). Every call shares the
 * array and its arrival counter: calls whose work overlaps on the GPU (for
 * example on two streams at once) race and must be serialised by the caller. */
hs_status hs_twist_noalloc(int L, const double* psi_dev, int K, double* z_dev,
                           void* cuda_stream);

/* Host-only: eigen-decomposition of the symmetric tridiagonal T (diagonal
 * alpha[0..k), off-diagonal beta[0..k-1)) by implicit QL with Wilkinson shifts.
 * theta[k] ascending; Y (k x k, column-major, may be NULL) eigenvectors.
 * Used for T_k of Algorithm 1. No GPU needed. */
hs_status hs_tridiag_eig(int k, const double* alpha, const double* beta, double* theta,
                         double* Y);

/* Derivatives of the twist overlaps of K eigenpairs with respect to the fields,
 * by the adjoint of first-order perturbation theory. For each eigenpair
 * (evals_host[i], psi_dev + i n) of H (real, non-degenerate; psi normalised by
 * the call), with z = <psi|U_twist|psi> (Sec. III) and dH/dh_j = -Sz_j (Eq. (1)):
 *   dz/dh_j = 2 lambda^T Sz_j psi,  (H - E) lambda = P (psi * u),  lambda _|_ psi,
 * P = I - psi psi^T, u the diagonal of U_twist: one complex solve per pair, by
 * the preconditioned MINRES of Algorithm 2 (FP64, row-norm preconditioner,
 * shift E, relative tolerance tol; <= 0: 1e-10), whatever the number of sites.
 * Outputs (host): z_host[2i], [2i+1] = Re, Im z_i (may be NULL);
 * dz2_host[i L + j] = d|z_i|^2 / dh_{j+1}; dE_host[i L + j] = dE_i / dh_{j+1}
 * = -<psi_i|Sz_{j+1}|psi_i> (Hellmann-Feynman; may be NULL); info: MINRES
 * iterations summed over the solves (may be NULL). The handle's sigma is
 * restored on return. Returns HS_NOT_CONVERGED if a solve reaches 50 n
 * iterations (the gradients of the pairs done so far are valid). */
hs_status hs_twist_grad(hs_handle* hd, const double* psi_dev, const double* evals_host, int K,
                        double tol, double* z_host, double* dz2_host, double* dE_host,
                        hs_minres_info* info);

/* Bipartite entanglement entropy S_i = -Tr rho_A log rho_A (natural logarithm)
 * of the K real FP64 vectors psi_dev + i n, n = C(L, L/2), for the subsystem A
 * of sites 1..L/2 (Sec. IV B). The vectors need not be normalised (rho_A is
 * divided by its trace). rho_A is block diagonal in the number a of up spins
 * of A; each block rho_a = Psi_a Psi_a^T (Psi_a: the C(L/2, a) x C(L/2, a)
 * coefficient block) is formed on the device in FP64, its eigenvalues on the
 * host (as hs_sym_eigvals, one host thread per block). S_host: K entropies.
 * Device scratch: sum_a C(L/2, a)^2 doubles (320 MB at L = 28), taken from
 * the handle's pool and returned. Synchronises the stream. */
hs_status hs_entanglement(hs_handle* hd, const double* psi_dev, int K, double* S_host);

/* Level spacing ratios of Sec. IV B: with the K eigenvalues sorted and
 * d_k = E_{k+1} - E_k, r_k = min(d_k, d_{k-1}) / max(d_k, d_{k-1}) for the
 * K - 2 interior levels (r_host, may be NULL; equal neighbouring gaps of zero
 * give 1), and *mean_out their mean (may be NULL). K >= 3, finite values.
 * Host-only. */
hs_status hs_level_ratio(const double* evals_host, int K, double* r_host, double* mean_out);

/* Host-only: eigenvalues w_host[n] (ascending) of the symmetric n x n matrix
 * a_host (row-major; both triangles read, overwritten) by Householder
 * reduction to tridiagonal form and implicit QL. The host step of
 * hs_entanglement. */
hs_status hs_sym_eigvals(int n, double* a_host, double* w_host);

/* Limit the persistent MINRES solves of this handle to nsm SMs (0 = all).
 * Independent handles on separate streams, each with a share of the SMs, then
 * solve their systems concurrently (several disorder realisations at once).
 * The share is read at the start of every MINRES solve, so another host thread
 * may change it while hs_lanczos_eigs runs on this handle: the new share takes
 * effect from the next Lanczos step (for example, to hand the SMs of finished
 * realisations to the ones still running). Keep the shares of concurrent
 * handles summing to at most the SM count. The paper runs one realisation per
 * GPU; this is a throughput setting only. */
hs_status hs_set_sm_budget(hs_handle* hd, int nsm);

/* Number of CUDA kernels this library has launched in the process so far
 * (every launch site increments it; graph replays count their kernels).
 * Host-only; used to report how many kernels a timed region ran. */
unsigned long long hs_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* HS_H */
