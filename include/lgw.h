/*
 * lgw.h - C ABI of the GB300 (sm_103a) Lanczos full-frequency GW hot path.
 *
 * Method: Gao, Tang, Zhao, Chelikowsky, "Efficient Full-frequency GW
 * Calculations using a Lanczos Method" (arXiv 2310.20103).
 *
 * The library computes the correlation self-energy Sigma^corr_tt(omega) of
 * Eq. 7 for a set of target orbitals t without diagonalising the reduced
 * Casida matrix (Eq. 4)
 *
 *     C = Delta^2 + c_K Delta^1/2 K Delta^1/2,   K = L L^T,
 *     Delta = diag(eps_c - eps_v)                (pair index vc = v*n_c + c)
 *
 * For every pair (t, m) of a target t and a summed orbital m it runs a
 * k-step Lanczos recurrence on C (Eq. 13) from the start vector |P_tm> of
 * the text after Eq. 8, b_tm = Delta^1/2 V_tm with (tm|vc) = V_tm[vc] =
 * sum_mu L[vc,mu] M_tm[mu], maps the tridiagonal's Gauss rule through
 * Omega = sqrt(theta) (Eq. 12, D = C^1/2), evaluates each term as a
 * continued fraction (Eq. 14) on a frequency grid, sums over m (Eq. 10) and
 * solves the quasiparticle equation E = eps_t + s_t + Re Sigma_t(E).
 *
 * Conventions shared by every call
 *   - Energies are in eV.  Complex outputs are interleaved (re, im) doubles.
 *   - A pointer argument may point to host memory or to device memory of the
 *     handle's device; the library detects which (cudaPointerGetAttributes)
 *     and copies host inputs in and host outputs out.  When any output is a
 *     host pointer the call returns only after the results are in place;
 *     otherwise it is asynchronous on the handle's stream and outputs are
 *     valid once that stream has been synchronised.
 *   - The caller owns every buffer it passes; no call keeps a caller pointer
 *     after it returns.  A system owns its own copies of eps, Delta and L.
 *     A handle owns the device workspace (Krylov basis, vector blocks) and
 *     grows it on demand; it is freed by lgw_destroy or
 *     lgw_release_workspace, and lgw_set_workspace_limit caps it.
 *   - Errors are return codes; nothing aborts and no exception crosses the
 *     ABI.  Device-side failures (non-positive Gauss nodes, a bounded wait
 *     that ran out) are collected in a device status word read at the end of
 *     a call.  lgw_last_error gives a one-line description of the last
 *     failure on a handle.  A handle is not thread-safe; use one per thread.
 */
#ifndef LGW_H
#define LGW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LGW_OK = 0,
  LGW_ERR_ARG = 1,             /* null pointer, negative size, bad enum      */
  LGW_ERR_SHAPE = 2,           /* inconsistent sizes or indices out of range */
  LGW_ERR_CUDA = 3,            /* a CUDA runtime call failed                 */
  LGW_ERR_OOM = 4,             /* device allocation failed                   */
  LGW_ERR_NOT_SPD = 5,         /* Delta <= 0 or a Gauss node theta <= 0      */
  LGW_ERR_NO_CONVERGENCE = 6,  /* tridiagonal eigensolver or QP solve failed */
  LGW_ERR_TIMEOUT = 7,         /* a bounded device wait ran out              */
  LGW_ERR_UNSUPPORTED = 8      /* option combination not built               */
} lgw_status;

/* Arithmetic of the two low-rank contractions L^T(Delta^1/2 X) and L Y.
 * Everything else (recurrence, reorthogonalisation, spectral map,
 * continued fractions, QP) is FP64 in every mode.  Start vectors V = L M
 * are FP64 in the FP64 mode and split BF16 (three products) otherwise. */
typedef enum {
  LGW_FP64 = 0,   /* FP64 CUDA-core GEMMs: the plain FP64 path            */
  LGW_BF16 = 1,   /* BF16 tcgen05 tensor-core GEMMs, FP32 accumulate      */
  LGW_FP8 = 3,    /* E4M3 tcgen05 GEMMs (kind::f8f6f4), FP32 accumulate:
                     L with one power-of-two scale per column (max -> (224,
                     448]), the per-step operands Delta^1/2 q and y with one
                     power-of-two scale per vector; 2 is reserved          */
  LGW_FP8_DEQ = 4 /* L in E4M3 as for LGW_FP8 (the same copies, half the
                     bytes of BF16), loaded by TMA and widened to FP16 in
                     shared memory (exact for every E4M3 value); the
                     per-step operands in FP16 with one power-of-two scale
                     per vector (largest value in (2^14, 2^15]); kind::f16
                     tcgen05 GEMMs, FP32 accumulate.  Only L is rounded to
                     8 bits.                                              */
} lgw_precision;

typedef enum {
  LGW_REORTH_NONE = 0,  /* three-term recurrence only                            */
  LGW_REORTH_CGS2 = 1,  /* full classical Gram-Schmidt, always two passes        */
  LGW_REORTH_CGS1K = 2, /* full CGS, second pass only where the norm drops below
                           1/sqrt(2) of its value before the pass (Kahan-Parlett
                           / Daniel-Gragg-Kaufman-Stewart criterion)              */
  LGW_REORTH_DCGS = 3   /* full CGS with the update delayed by one step: the
                           projection coefficients of w_j are computed in step
                           j, and q_{j+1} = (w_j - Q_j h_j)/beta_{j+1} is formed
                           in step j+1 inside the same single pass over the
                           stored basis that computes w_{j+1}'s coefficients
                           (one read of the basis per step instead of two).
                           The contractions of step j+1 run on w_j/beta_{j+1};
                           the difference C Q_j h_j/beta lies in span(Q_j) plus
                           a multiple of q_{j+1} and is removed by the same
                           projection, whose q_{j+1} coefficient is corrected
                           by h_{j,j} in the recorded alpha_{j+1}.  A second
                           pass is taken where the norm drops below 1/sqrt(2),
                           as in CGS1K.  Split (float-pair / float) basis only;
                           with the FP64 basis it runs as CGS1K.            */
} lgw_reorth;

/* Arithmetic of the full reorthogonalisation.
 * LGW_RA_FP64:  basis stored in FP64, every product and sum on the FP64 pipe.
 * LGW_RA_SPLIT: basis stored as float pairs (hi + lo, 48 significant bits);
 *               dot products in double-float arithmetic on the FP32 pipe; the
 *               update applies the two O(||w||) coefficients (q_j, q_{j-1}) in
 *               FP64 and the O(eps||w||) rest in FP32 from the hi part.
 *               Orthogonality stays at FP64 level; the FP64 pipe, which runs at
 *               1/58 of the FP32 rate on GB300, leaves the inner loops.
 * LGW_RA_SPLIT32: as SPLIT but only the hi float of each basis vector is
 *               stored and read (4 instead of 8 bytes per element in the dot
 *               products).  Products with the FP64 w stay exact; w ends up
 *               orthogonal to fl32(q_i), i.e. within ~2^-24 / sqrt(N_vc) of
 *               orthogonal to q_i (about 1e-10 at N_vc = 131072), inside the
 *               semi-orthogonality (sqrt(eps)) that keeps T_k accurate.
 * LGW_RA_AUTO:  SPLIT with BF16 contractions, FP64 with FP64 contractions. */
typedef enum {
  LGW_RA_AUTO = 0,
  LGW_RA_FP64 = 1,
  LGW_RA_SPLIT = 2,
  LGW_RA_SPLIT32 = 3
} lgw_reorth_arith;

typedef struct lgw_handle lgw_handle;
typedef struct lgw_system lgw_system;

/* Which copies of L a system keeps (lgw_system_desc.flags, OR-ed).
 *   LGW_SYS_NO_FP64  no padded FP64 copy: precision LGW_FP64,
 *                    lgw_sigma_c_backward and FP64 start vectors are then
 *                    LGW_ERR_UNSUPPORTED (start vectors from M use the split-
 *                    BF16 tensor-core product, so the BF16 copies are needed)
 *   LGW_SYS_NO_BF16  no BF16 copies (L, L^T, low half): precision LGW_BF16
 *                    is unsupported; start vectors from M use the FP64 copy
 *   LGW_SYS_FP8      make the E4M3 copies now (otherwise on the first FP8 or FP8_DEQ
 *                    request; with LGW_SYS_NO_FP64 they are always made now)
 * Every copy is made straight from desc->L, so a caller may free its L once
 * lgw_prepare_system has returned (device memory at N_vc = 1.6M, N_aux =
 * 8192: FP64 copy 105 GB, BF16 copies 79 GB, E4M3 copies 26 GB). */
enum {
  LGW_SYS_NO_FP64 = 1,
  LGW_SYS_NO_BF16 = 2,
  LGW_SYS_FP8 = 4
};

/* One electronic system: KS energies and the Coulomb-kernel factor.
 * eps  [n_v + n_c]          valence block first (Eq. 1-3: v occupied, c empty)
 * L    [n_v*n_c][n_aux]     row-major, K = L L^T (Eq. 15-17 fitted form)
 * kernel_factor             c_K in C = Delta^2 + c_K Delta^1/2 K Delta^1/2;
 *                           4.0 for a closed-shell spin sum, 0 switches K off.
 * flags                     LGW_SYS_* (0: FP64 and BF16 copies, E4M3 on use) */
typedef struct {
  int32_t n_v, n_c, n_aux;
  const double *eps;
  const double *L;
  double kernel_factor;
  int32_t flags;
} lgw_system_desc;

/* The self-energy request.
 * targets [n_t]   orbital indices t (diagonal elements Sigma_tt, Eq. 5-7)
 * m_idx   [n_m]   summed orbital indices m (Eq. 10; a subset is allowed)
 * M  [n_t][n_m][n_aux]  fitting factors: (tm|vc) = sum_mu L[vc,mu] M[t,m,mu]
 * V  [n_t][n_m][n_v*n_c] the couplings (tm|vc) directly
 *                 exactly one of M and V is non-NULL
 * omega [n_freq]  real frequency grid; delta > 0 the broadening of Eq. 7
 * static_shift [n_t] or NULL: s_t in E = eps_t + s_t + Re Sigma_t(E)
 *                 (exchange minus exchange-correlation potential; 0 if NULL) */
typedef struct {
  int32_t n_t;
  const int32_t *targets;
  int32_t n_m;
  const int32_t *m_idx;
  const double *M;
  const double *V;
  int32_t n_freq;
  const double *omega;
  double delta;
  const double *static_shift;
} lgw_problem;

/* k              Lanczos steps per start vector (1 <= k <= n_v*n_c)
 * precision      lgw_precision of the two contractions
 * reorth         lgw_reorth
 * b_sub          start vectors per sub-batch (0: automatic)
 * breakdown_tol  a vector stops after step j when beta_{j+1} <= tol*max|alpha|
 *                (0: 1e-13)
 * qp_max_iter    Newton iterations before the bracketing fallback (0: 50)
 * qp_tol         |dE| <= qp_tol * max(1,|E|) ends Newton (0: 1e-10)
 * use_graph      1: capture each sub-batch's launch sequence (start vectors
 *                and the k Lanczos steps) as a CUDA graph on first use and
 *                replay it from a per-handle cache when the same system,
 *                shapes, options and buffers come again; the report's
 *                per-category times are then zero (ms_total stays)
 * reorth_arith   arithmetic of the Gram-Schmidt passes (lgw_reorth_arith)
 * qp_mode        0: graphical solution of E = eps_t + s_t + Re Sigma_t(E)
 *                (Newton, bracketing fallback); 1: linearised at e0 = eps_t +
 *                s_t, E = e0 + Z Re Sigma_t(e0), Z = 1 / (1 - Re Sigma_t'(e0))
 * ckpt_every     backward calls, FP64 without reorthogonalisation: steps
 *                between Krylov checkpoints of the exact reverse sweep
 *                (0: 16; the forward keeps q_{s-1}, q_s at every multiple s
 *                of it and recomputes the steps in between) */
typedef struct {
  int32_t k;
  int32_t precision;
  int32_t reorth;
  int32_t b_sub;
  double breakdown_tol;
  int32_t qp_max_iter;
  double qp_tol;
  int32_t use_graph;
  int32_t reorth_arith;
  int32_t qp_mode;
  int32_t ckpt_every;
} lgw_options;

/* Filled by calls that take a report pointer (host memory).  Phase times are
 * sums of CUDA-event intervals on the handle's stream; asking for a report
 * makes the call record those events and synchronise at its end. */
typedef struct {
  double ms_total;
  double ms_start;       /* coupling/start vectors and first normalisation   */
  double ms_gemm1;       /* L^T (Delta^1/2 q) contraction + partial reduce   */
  double ms_gemm2;       /* L y contraction + fused recurrence epilogue      */
  double ms_dots;        /* alpha finish, axpy and first-pass Q^T w products
                            (LGW_REORTH_DCGS: the single sweep)             */
  double ms_update;      /* first-pass w -= Q h (with the split basis also
                            q_{j+1} for vectors that take no second pass;
                            LGW_REORTH_DCGS: the per-vector reduction)      */
  double ms_pass2;       /* second Gram-Schmidt pass (decision, Q^T w, update) */
  double ms_normalize;   /* beta, breakdown test, q_{j+1}, bf16 operand (0
                            with the split basis: folded into the update)   */
  double ms_spectral;    /* tridiagonal eigenproblems and Jacobi rebuild     */
  double ms_cf;          /* continued fractions on the grid                  */
  double ms_qp;          /* quasiparticle solve                              */
  double gemm_flops;     /* algorithmic 4 N_vc N_aux k per vector, summed    */
  double reorth_elems;   /* basis elements visited per Gram-Schmidt kernel,
                            sum over vectors of N_vc * sum_j (j+1)            */
  int32_t n_vectors;     /* start vectors B = n_t n_m                        */
  int32_t n_sub_batches;
  int32_t b_sub;         /* padded vectors per sub-batch                     */
  int32_t k_min, k_max;  /* effective Lanczos depth over vectors             */
  int32_t n_second_pass; /* vector-steps that took a second CGS pass         */
  int32_t gpu_launches;  /* kernels launched by the call                     */
  int32_t gemm1_splits;  /* K splits of the first contraction                */
  double min_theta;      /* smallest Gauss node over all tridiagonals        */
} lgw_report;

/* Status text for a code; never NULL. */
const char *lgw_status_string(lgw_status s);

/* Create a handle bound to CUDA device `device` and the CUDA stream
 * `cuda_stream` (a cudaStream_t; NULL means the legacy default stream).
 * Allocates only the status word. */
lgw_status lgw_create(lgw_handle **out, int device, void *cuda_stream);

/* Destroy a handle and free its workspace.  Systems created on it must be
 * released first.  NULL is accepted. */
lgw_status lgw_destroy(lgw_handle *h);

/* Copy the last error message of `h` into buf (NUL-terminated, truncated to
 * n bytes).  Returns the last error code. */
lgw_status lgw_last_error(lgw_handle *h, char *buf, size_t n);

/* Workspace budget (the paper has no counterpart; a service for callers that
 * share a GPU).  lgw_set_workspace_limit caps the device bytes the handle's
 * workspace may hold (0: no cap, the default).  A call whose next
 * workspace allocation would pass the cap returns LGW_ERR_OOM before that
 * allocation; nothing already held is freed and the handle stays usable
 * (work queued earlier in the call completes on valid buffers).  A failed
 * cudaMalloc gives LGW_ERR_OOM the same way.  lgw_workspace_bytes reports
 * the bytes held; lgw_release_workspace waits for the handle's stream and
 * frees the whole workspace (later calls allocate it again). */
lgw_status lgw_set_workspace_limit(lgw_handle *h, size_t bytes);
lgw_status lgw_workspace_bytes(lgw_handle *h, size_t *bytes);
lgw_status lgw_release_workspace(lgw_handle *h);

/* Diagnostic of the bounded device waits (the paper has no counterpart).
 * Every wait of the library's kernels on an mbarrier phase (the tensor-core
 * pipeline's TMA and MMA hand-offs) gives up after a cycle limit, sets a
 * timeout bit in the handle's status word and lets the kernel finish, so
 * the context stays usable and the call returns LGW_ERR_TIMEOUT.  This call
 * runs that same wait once, in one small kernel, with a limit of `seconds`
 * (1e-4 .. 2): with arrive != 0 another thread completes the barrier first
 * and the call returns LGW_OK; with arrive == 0 nothing ever completes it,
 * the wait runs out and the call returns LGW_ERR_TIMEOUT.  No copy or other
 * asynchronous operation is in flight during the wait.  Synchronous. */
lgw_status lgw_selftest_bounded_wait(lgw_handle *h, int32_t arrive, double seconds);

/* Build a system: copies eps to the device, forms Delta_vc, Delta^1/2 and
 * Delta^2 (Eq. 2-4), and makes the copies of L that desc->flags asks for,
 * each padded to [N_pad][A_pad]: FP64, BF16 (L, L^T and the low half
 * bf16(L - bf16(L))) and E4M3 (L, L^T, column scales).
 * Fails with LGW_ERR_NOT_SPD if some eps_c - eps_v <= 0 and with
 * LGW_ERR_ARG for unknown flags or LGW_SYS_NO_FP64 | LGW_SYS_NO_BF16. */
lgw_status lgw_prepare_system(lgw_handle *h, const lgw_system_desc *desc, lgw_system **out);

/* Free a system's device memory.  NULL is accepted. */
lgw_status lgw_release_system(lgw_system *s);

/* Apply C to n_vec vectors: Y[i] = C X[i], X and Y [n_vec][n_v*n_c] FP64,
 * through the same contractions (precision) the Lanczos path uses. */
lgw_status lgw_apply_casida(lgw_handle *h, const lgw_system *s, int32_t n_vec,
                            const double *X, double *Y, int32_t precision);

/* Lanczos tridiagonals only (Eq. 13) for every start vector, vector index
 * i = t_index * n_m + m_index:
 *   alpha [B][k]  diagonal a_0..a_{k-1}
 *   beta  [B][k]  beta[i][j] couples steps j and j+1; beta[i][k-1] is the
 *                 final residual norm
 *   beta0 [B]     ||b_tm||
 *   k_eff [B]     steps actually taken (< k after a breakdown)
 * These arrays are a complete checkpoint: lgw_sigma_from_coeffs resumes
 * from them. */
lgw_status lgw_lanczos_coeffs(lgw_handle *h, const lgw_system *s, const lgw_problem *p,
                              const lgw_options *o, double *alpha, double *beta,
                              double *beta0, int32_t *k_eff);

/* Self-energy and QP energies from stored tridiagonals (Eq. 12, 14, 10):
 * spectral map of each T_k, continued fractions on the grid, QP solve.
 * sigma [n_t][n_freq][2]; e_qp [n_t]; z_qp [n_t] (renormalisation factor
 * 1/(1 - dRe Sigma/domega) at E_qp) may be NULL.  Orbital indices are
 * checked on the host; a depth k_eff outside [0, k] makes the spectral map
 * skip that vector and the call return LGW_ERR_SHAPE. */
lgw_status lgw_sigma_from_coeffs(lgw_handle *h, const lgw_system *s, const lgw_problem *p,
                                 const lgw_options *o, const double *alpha,
                                 const double *beta, const double *beta0,
                                 const int32_t *k_eff, double *sigma, double *e_qp,
                                 double *z_qp);

/* The whole hot path for one system: start vectors, k Lanczos steps per
 * (t, m) pair, spectral map, continued fractions on the grid (Eq. 14, one
 * thread per (target, frequency)), sum over m (Eq. 10) and QP solve.
 * sigma [n_t][n_freq][2], e_qp [n_t], z_qp [n_t] or NULL, rep or NULL. */
lgw_status lgw_sigma_c(lgw_handle *h, const lgw_system *s, const lgw_problem *p,
                       const lgw_options *o, double *sigma, double *e_qp, double *z_qp,
                       lgw_report *rep);

/* The paper's polynomial form (text after Eq. 12): D = p_g(C) ~ C^1/2 with
 * p_g the degree-g Chebyshev interpolant of sqrt at the g+1 Chebyshev points
 * of the first kind on [x_lo, x_hi] (the spectral interval of C: x_lo <=
 * lambda_min, x_hi >= lambda_max; eps_c - eps_v bounds lambda_min from
 * below), Lanczos on D from each |P_tm> (Eq. 13; D applied by Clenshaw's
 * recurrence, g applications of C per step, FP64 Krylov basis), and
 * Sigma_tm(omega) = (1/z) <P|D^-1 - (D + eta z)^-1|P> from two Haydock
 * continued fractions of D's tridiagonal (Eq. 14), z = omega - eps_m - i eta
 * delta.  Outputs as lgw_sigma_c; the report's gemm_flops count g products
 * per step.  x_lo = x_hi = 0 asks the library for the interval
 * (lgw_spectral_interval with k = 32; estimated once per system, on the
 * first such call, with one synchronisation, then kept with the system). */
typedef struct {
  int32_t g;           /* degree, 1..256 */
  double x_lo, x_hi;   /* 0 < x_lo < x_hi, or both 0 */
} lgw_poly;

/* Interval [x_lo, x_hi] around the spectrum of C for the polynomial fit
 * (the text after Eq. 12 fits p_g on the range of C's eigenvalues):
 *   x_lo = min over pairs of Delta^2 = (eps_c - eps_v)^2, a lower bound of
 *          lambda_min because C = Delta^2 + c_K Delta^1/2 L L^T Delta^1/2
 *          adds a positive semidefinite term;
 *   x_hi = the largest Ritz value of k Lanczos steps (Eq. 13, CGS2; BF16
 *          tensor-core contractions when the system has its BF16 copies,
 *          else FP64)
 *          from a fixed pseudo-random start vector, plus that step's beta,
 *          the residual norm, which bounds the distance from the Ritz value
 *          to an eigenvalue of C.  The largest Ritz value converges to
 *          lambda_max from below first; x_hi is an estimate, not a bound.
 * Host outputs; synchronous.  LGW_ERR_NOT_SPD if the estimate is not a
 * positive interval. */
lgw_status lgw_spectral_interval(lgw_handle *h, const lgw_system *s, int32_t k, double *x_lo,
                                 double *x_hi);

lgw_status lgw_sigma_c_poly(lgw_handle *h, const lgw_system *s, const lgw_problem *p,
                            const lgw_options *o, const lgw_poly *poly, double *sigma,
                            double *e_qp, double *z_qp, lgw_report *rep);

/* Tridiagonals of D = p_g(C) only (as lgw_lanczos_coeffs). */
lgw_status lgw_lanczos_coeffs_poly(lgw_handle *h, const lgw_system *s, const lgw_problem *p,
                                   const lgw_options *o, const lgw_poly *poly, double *alpha,
                                   double *beta, double *beta0, int32_t *k_eff);

/* Self-energy matrix Sigma_tt'(omega) of the request's targets (n_t = p,
 * 1..8) by band Lanczos: the band method for matrix elements of a resolvent
 * that the paper cites after Eq. 14, here with the square-root map of the
 * Gauss rule (Eq. 12) in place of the resolvent of D.  For each summed
 * orbital m one recurrence starts from the block [b_{t,m} over the
 * targets], orthonormalised into q_0..q_{p-1} with b_t = sum_i R0[i][t] q_i;
 * step j applies C to q_j (one matvec per m and step, through the same
 * contractions as lgw_sigma_c) and projects the result out of all of m's
 * basis vectors twice (classical Gram-Schmidt, FP64 basis), giving column j
 * of the banded T = Q^T C Q and at most one new basis vector.  The k x k T
 * then yields every element b_t . f(C) b_t' with f(theta) =
 * 1/(sqrt(theta)(z_m + eta_m sqrt(theta))): a k-step Lanczos on T from
 * R0 e_t (diagonal) and from R0 (e_t +- e_t') (pairs, combined by the
 * polarisation identity), each mapped and summed like lgw_sigma_c's
 * fractions (Eq. 7, 10-14).  This shares one recurrence per m among all
 * p(p+1)/2 elements, where lgw_sigma_offdiag runs two per pair.  Exact once
 * the block Krylov space is exhausted.
 *   sigma [n_t][n_t][n_freq][2] (symmetric); rep or NULL.
 * Limits: precision FP64 or BF16 (LGW_ERR_UNSUPPORTED for either E4M3 mode), k <= 512;
 * o->reorth is not used (always two projections); the static shift and QP
 * options are not used.  Scratch: k^2 doubles per (m, element vector). */
lgw_status lgw_sigma_band(lgw_handle *h, const lgw_system *s, const lgw_problem *p,
                          const lgw_options *o, double *sigma, lgw_report *rep);

/* Exchange self-energy Sigma^ex_t = -sum_v (vt|vt) (text after Eq. 5) over
 * the occupied orbitals v of the request's summed set, from its pair factors
 * (which share L's metric-folded form, (pq|rs) = sum_mu B_pq,mu B_rs,mu):
 * (vt|vt) = sum_mu M[t][v][mu]^2.  p->M is required (LGW_ERR_UNSUPPORTED with
 * V).  sigma_x [n_t], host or device.  With a V_xc of the caller,
 * static_shift = sigma_x - V_xc turns the QP equation into the full one. */
lgw_status lgw_sigma_x(lgw_handle *h, const lgw_system *s, const lgw_problem *p,
                       double *sigma_x);

/* Density-fitting factors: with fitting coefficients C [n_pairs][n_aux] of
 * orbital pairs and the Coulomb metric [n_aux][n_aux] (symmetric positive
 * definite), (ab|cd) = sum C_ab,mu metric_mu,nu C_cd,nu = sum_kappa B_ab,kappa
 * B_cd,kappa with B = C R, metric = R R^T (FP64 blocked Cholesky and FP64
 * product on the GPU).  B [n_pairs][n_aux]; the factors of the vc pairs are
 * the system's L, those of the (t, m) pairs the request's M.  Host or device
 * pointers; LGW_ERR_NOT_SPD if the metric is not positive definite. */
lgw_status lgw_fit_factors(lgw_handle *h, int32_t n_pairs, int32_t n_aux, const double *C,
                           const double *metric, double *B);

/* Tamm-Dancoff variant (B = 0 in Eq. 1): the excitations are the eigenpairs
 * of A = Delta + (c_K / 2) L L^T (A carries the kernel once, A + B twice)
 * and W^s_tm = sum_vc (tm|vc) X^s_vc, so Sigma_tm(omega) = V^T (z + eta A)^-1 V
 * = -eta G(-eta z) with G the Haydock fraction of A's own k-step tridiagonal
 * started from V = L M (Eq. 13-14; no square-root map).  Options, outputs and
 * precisions as lgw_sigma_c; the adjoint is not available for it. */
lgw_status lgw_sigma_c_tda(lgw_handle *h, const lgw_system *s, const lgw_problem *p,
                           const lgw_options *o, double *sigma, double *e_qp, double *z_qp,
                           lgw_report *rep);

/* Off-diagonal elements Sigma_tt'(omega) = sum_m sum_s W^s_tm W^s_t'm /
 * (Omega_s (z + eta Omega_s)) (Eq. 7) for n_pairs pairs (t, t') given as
 * indices into p->targets (pairs [n_pairs][2], host or device), by the
 * polarisation identity over diagonal elements:
 *   Sigma_tt' = (Sigma[b_t + b_t'] - Sigma[b_t - b_t']) / 4,
 * i.e. 2 n_pairs requests whose factors are M_t +- M_t' (or V_t +- V_t').
 * sigma_od [n_pairs][n_freq][2]; no QP solve. */
lgw_status lgw_sigma_offdiag(lgw_handle *h, const lgw_system *s, const lgw_problem *p,
                             const lgw_options *o, int32_t n_pairs, const int32_t *pairs,
                             double *sigma_od);

/* Several independent systems of uneven size in one call; sigma[i], e_qp[i]
 * and z_qp[i] (z_qp may be NULL) have the shapes of lgw_sigma_c for
 * problems[i].  The systems run concurrently on up to four internal streams
 * (system i on stream i % 4, each stream with its own workspace, so the
 * device memory held is up to four single-system workspaces); the call
 * orders itself after earlier work on the handle's stream and later work on
 * that stream after itself.  Results equal one lgw_sigma_c per system.
 * With rep, ms_total covers the whole call and the per-category times are
 * zero (the systems overlap). */
lgw_status lgw_sigma_c_batched(lgw_handle *h, int32_t n_sys, const lgw_system *const *systems,
                               const lgw_problem *problems, const lgw_options *o,
                               double *const *sigma, double *const *e_qp,
                               double *const *z_qp, lgw_report *rep);

/* Allocation-free variant of lgw_sigma_from_coeffs (the paper has no
 * counterpart; this is a service for callers).
 *
 * Some callers cannot let a library allocate device memory while they run:
 * services that give the library a fixed device-memory budget at start-up,
 * or latency-bound loops where cudaMalloc/cudaFree would synchronise the
 * device and stall other streams.  This call computes exactly what
 * lgw_sigma_from_coeffs computes -- spectral map, continued fractions on the
 * grid, QP solve -- without any allocation: its scratch is one static device
 * array of 16 MiB (2^21 doubles) that every GPU loading the library holds
 * until the process exits.
 *
 * Requirements and limits
 *   - every array (alpha, beta, beta0, k_eff, sigma, e_qp, z_qp if given, and
 *     p->targets, p->m_idx, p->omega, p->static_shift if given) must be
 *     device memory of the handle's device; host pointers and memory of
 *     another device give LGW_ERR_ARG.  p->M and p->V are not used.  sigma
 *     and e_qp are required.
 *   - B = n_t * n_m vectors with k steps need B * (5k + 2) + 1 doubles; larger
 *     requests are rejected with LGW_ERR_UNSUPPORTED and nothing runs.
 *     k above 4095 gives LGW_ERR_UNSUPPORTED and an unknown qp_mode
 *     LGW_ERR_ARG, both before any launch.
 *   - an orbital index outside [0, n_v + n_c) in p->targets or p->m_idx, or
 *     a depth k_eff outside [0, k], gives LGW_ERR_SHAPE.  The arrays live on
 *     the device, so a first kernel checks them and the call reads its
 *     verdict back (one stream synchronisation) before it queues any kernel
 *     that uses an index; on failure nothing else runs.
 *   - the first call on a device looks up the device address of the static
 *     array (cudaGetSymbolAddress); make that first call before any stream
 *     capture on that device.
 *   - all calls share the one array and overwrite it; calls whose work
 *     overlaps on the GPU (several streams or handles at once) race and give
 *     undefined results.  The call returns after its stream has finished. */
lgw_status lgw_sigma_from_coeffs_noalloc(lgw_handle *h, const lgw_system *s,
                                         const lgw_problem *p, const lgw_options *o,
                                         const double *alpha, const double *beta,
                                         const double *beta0, const int32_t *k_eff,
                                         double *sigma, double *e_qp, double *z_qp);

/* Gradient of sum_t dE[t] * E_qp[t] with respect to L ([n_v*n_c][n_aux]) and
 * eps ([n_v+n_c]) for the request p, through the adjoint of the Lanczos
 * recurrence (Eq. 13), the spectral map and Gauss rule (Eq. 12, 14), the
 * continued fractions and the QP equation (graphical solution, qp_mode 0;
 * implicit-function factor Z_t).  dL / deps are overwritten; either may be
 * NULL.  Two forms:
 *   - precision LGW_FP64 with reorth LGW_REORTH_NONE: the exact derivative
 *     of the k-step energies, by reverse mode of the three-term recurrence.
 *     The forward keeps Krylov checkpoints every o->ckpt_every steps (0: 16)
 *     and each segment is recomputed before it is taken back, so device
 *     memory holds 2 k / ckpt_every + 2 ckpt_every + 12 vectors per start
 *     vector instead of the k + 1 of a stored basis.
 *   - otherwise (full reorthogonalisation, or BF16/E4M3 contractions): the
 *     Krylov form over the stored basis, dF/db = Q a, dF/dC = Q Gam Q^T with
 *     the Daleckii-Krein coefficients of T_k.  Exact at k = n_v*n_c; at
 *     truncated k it approximates the derivative of the k-step energies to
 *     the accuracy with which those energies have converged in k.
 * qp_mode 1 gives LGW_ERR_UNSUPPORTED; a negative ckpt_every LGW_ERR_ARG. */
lgw_status lgw_sigma_c_backward(lgw_handle *h, const lgw_system *s, const lgw_problem *p,
                                const lgw_options *o, const double *dE, double *dL,
                                double *deps);

/* The same gradient for the Tamm-Dancoff energies of lgw_sigma_c_tda
 * (A = Delta + c_K/2 L L^T, b = V = L M, f(theta) = 1/(z + eta theta); the
 * text after Eq. 4 and Eq. 7 with the resonant block alone):
 * dL = c_K G L + y M^T, dDelta = diag(G).  Same two forms and limits. */
lgw_status lgw_sigma_c_tda_backward(lgw_handle *h, const lgw_system *s, const lgw_problem *p,
                                    const lgw_options *o, const double *dE, double *dL,
                                    double *deps);

/* The same gradient for the polynomial form of lgw_sigma_c_poly (Lanczos on
 * D = p_g(C), the fit of sqrt after Eq. 12; fractions on D's tridiagonal,
 * Eq. 14).  Exact form only: o->precision LGW_FP64 and o->reorth
 * LGW_REORTH_NONE (otherwise LGW_ERR_UNSUPPORTED).  Each step is taken back
 * through the reverse of Clenshaw's recurrence, so a step costs 3 g
 * products with C besides the forward's g.  The interval [x_lo, x_hi] is a
 * fixed input: with x_lo = x_hi = 0 the library's own estimate (as in
 * lgw_sigma_c_poly) is used and its dependence on L and eps is not part of
 * the gradient. */
lgw_status lgw_sigma_c_poly_backward(lgw_handle *h, const lgw_system *s, const lgw_problem *p,
                                     const lgw_options *o, const lgw_poly *poly,
                                     const double *dE, double *dL, double *deps);

#ifdef __cplusplus
}
#endif

#endif /* LGW_H */
