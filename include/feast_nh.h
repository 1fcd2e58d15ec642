/*
 * feast_nh.h - C ABI of the GB300 (sm_103a) non-Hermitian FEAST hot path.
 *
 * Method: Kestyn, Polizzi, Tang, "FEAST eigensolver for non-Hermitian
 * problems".  For a pencil (A, B) and a contour C the library computes the
 * eigenvalues inside C with B-bi-orthonormal right and left eigenvectors,
 *     A X = B X Lambda,   A^H X^ = B^H X^ Lambda^*,   X^^H B X = I,
 * by subspace iteration with the contour-integration filter
 *     Q  = sum_j w_j   (z_j B - A)^{-1}   B   Y        (eq. qr)
 *     Q^ = sum_j w_j^* (z_j B - A)^{-H}   B^H Y^       (eq. ql)
 * followed by the B-bi-orthonormal Rayleigh-Ritz step (Fig. alg:three).
 *
 * Conventions shared by every entry point
 *  - Matrices are CSR, 0-based, int32 row pointers and column indices, held
 *    in DEVICE memory owned by the caller; they must stay valid and unchanged
 *    until feast_nh_destroy.  Column indices within a row need not be sorted;
 *    duplicates are summed.
 *  - Dense blocks (Y, Y^, Q, Q^, X, X^) are DEVICE arrays of complex double
 *    (interleaved re, im), ROW-major n x m with leading dimension m: entry
 *    (i, c) is at index i*m + c, i.e. a C-contiguous torch tensor of shape
 *    (n, m) and dtype complex128.  The caller owns them.
 *  - Small outputs `lambda` (complex, 2 doubles per entry) and `res` are
 *    DEVICE arrays of length m0; counts and the info struct are HOST memory.
 *  - All work is enqueued on the stream given to feast_nh_init.  feast_nh_filter,
 *    feast_nh_rr and feast_nh_solve read a few numbers back from the device
 *    (inner residual and error word, subspace size, counts, convergence flag)
 *    once per call / per outer iteration / per refinement step.
 *  - The library allocates its workspace in feast_nh_init (and, for the
 *    banded factors, on the first filter) and frees it in feast_nh_destroy.
 *  - Errors are returned, never raised or aborted; feast_nh_last_error gives
 *    a message for the last failing call on a context.  On FEAST_NH_ENOCONV
 *    the outputs hold the best iterate; on EINVAL/ECUDA they are undefined.
 */
#ifndef FEAST_NH_H
#define FEAST_NH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct feast_nh_ctx feast_nh_ctx; /* opaque, owned by the library */

typedef enum {
  FEAST_NH_OK = 0,
  FEAST_NH_EINVAL = 1,    /* bad argument (size, pointer, option)            */
  FEAST_NH_ENOMEM = 2,    /* device allocation failed                        */
  FEAST_NH_ECUDA = 3,     /* a CUDA call failed                              */
  FEAST_NH_ENOCONV = 4,   /* outer iteration cap reached: best iterate kept  */
  FEAST_NH_EINNER = 5,    /* inner solve did not reach its tolerance         */
  FEAST_NH_ESINGULAR = 6, /* zero pivot (node on an eigenvalue) or B_Q == 0  */
  FEAST_NH_ETIMEOUT = 7   /* a bounded device wait gave up                   */
} feast_nh_status;

typedef enum { FEAST_NH_R64 = 0, FEAST_NH_C64 = 1 } feast_nh_dtype;

/* CSR matrix in device memory (Sec. 3: sparse CSR driver). */
typedef struct {
  int32_t n;              /* order                                     */
  int64_t nnz;            /* number of stored entries                  */
  const int32_t *rowptr;  /* n+1 entries                               */
  const int32_t *colind;  /* nnz entries                               */
  const void *val;        /* nnz doubles (R64) or 2*nnz doubles (C64)  */
  int32_t dtype;          /* feast_nh_dtype                            */
} feast_nh_csr;

/* Search contour (Sec. 2.1).  kind 0: circle |z - c| = r.  kind 1: ellipse
 * z = c + e^{i angle}(r cos t + i ratio*r sin t).  kind 2: custom nodes and
 * weights z[2*ne], w[2*ne] (HOST arrays of interleaved complex doubles).
 * Kinds 0 and 1 use the trapezoidal rule with ne half-offset nodes
 * t_j = pi(2j-1)/ne and weights w_j = z'(t_j)/(i ne) (Sec. 2.3). */
typedef struct {
  int32_t kind;
  double c_re, c_im, r, ratio, angle;
  int32_t ne;
  const double *z, *w;
} feast_nh_contour;

enum { FEAST_NH_INNER_BANDED = 0, FEAST_NH_INNER_BICGSTAB = 1, FEAST_NH_INNER_FGMRES = 2 };
enum { FEAST_NH_PRECOND_NONE = 0, FEAST_NH_PRECOND_JACOBI = 1, FEAST_NH_PRECOND_LEARNED = 2 };
enum { FEAST_NH_PREC_FP64 = 0, FEAST_NH_PREC_FP32_IR = 1 };
enum { FEAST_NH_PROJ_FP64 = 0, FEAST_NH_PROJ_TENSOR = 1 };
enum { FEAST_NH_PROBLEM_GENERAL = 0, FEAST_NH_PROBLEM_COMPLEX_SYMMETRIC = 1 };

/* Options.  eps, eta, mu: eq. (res), eq. (resize), Sec. 2.7.  inner_tol is
 * the relative 2-norm residual each shifted solve must reach (iterative
 * refinement for FP32_IR, Krylov tolerance for BICGSTAB); inner_max caps
 * the refinement steps / Krylov iterations. */
typedef struct {
  double eps;         /* 1e-10  */
  double eta;         /* 1e-16  */
  double mu;          /* 0.1    */
  double inner_tol;   /* 1e-10  */
  int32_t max_iter;   /* 100    */
  int32_t inner_max;  /* 12     */
  int32_t inner_kind; /* FEAST_NH_INNER_BANDED */
  int32_t precision;  /* FEAST_NH_PREC_FP64    */
  int32_t problem;    /* FEAST_NH_PROBLEM_GENERAL */
  int32_t timing;     /* 1: record CUDA events around the banded solve and
                         multi-shift kernels; totals go to feast_nh_info   */
  int32_t krylov_max; /* 1000: Krylov iterations per refinement step (batched
                         solver and FGMRES)                                 */
  int32_t krylov_restart; /* 30: FGMRES restart length (<= 64)              */
  int32_t precond;    /* FGMRES right preconditioner: FEAST_NH_PRECOND_JACOBI
                         (default), _NONE, or _LEARNED (feast_nh_set_network) */
  int32_t projection; /* FEAST_NH_PROJ_TENSOR (default): the n x m^2 products
                         of the Rayleigh-Ritz step (B_Q, A_U, B_U of steps 2.a
                         and 4.a, U and Y of eq. uu and step 4.d) on the
                         tensor cores as exact products of integer digits
                         (FP64-accurate, see feast_nh_gram); FEAST_NH_PROJ_FP64:
                         FP64 arithmetic on the CUDA cores                  */
} feast_nh_opts;

/* Per-call record (host).  Times are CUDA-event milliseconds on the stream. */
typedef struct {
  int32_t iterations;   /* outer iterations done                              */
  int32_t m_tilde;      /* subspace size after the last resize                */
  int32_t m_r;          /* Ritz values inside C at the last iteration         */
  int32_t m_s;          /* of those, flagged spurious                         */
  int32_t m;            /* converged pairs returned (m_r - m_s)               */
  int32_t inner_steps;  /* refinement steps / Krylov iterations, last filter  */
  int32_t converged;    /* 1 if eq. (res) < eps for the m lowest residuals     */
  int32_t kl, ku;       /* band of (z B - A) found by the banded inner solver */
  double max_res;       /* largest of the m lowest residuals                  */
  double inner_res;     /* largest relative inner residual, last filter       */
  double t_factor_ms, t_filter_ms, t_rr_ms, t_total_ms;
  /* with opts.timing: summed device time and launch count of the banded
   * triangular-solve kernel and of the multi-shift residual kernel */
  double t_solve_kernel_ms, t_resid_kernel_ms;
  int32_t n_solve_launches, n_resid_launches;
  int32_t n_factorizations; /* shifted matrices factorised: ne, or ne/2 for a
                               real pencil whose nodes come in conjugate pairs
                               (Sec. 2.4, Table tab:solve)                    */
  int32_t inner_fail;       /* filters of this solve whose shifted solves
                               stopped above their tolerance (refinement or
                               Krylov cap reached)                            */
  double pivot_min, pivot_max; /* smallest / largest pivot modulus |u_rr| of
                               the banded factors (no pivoting is done: a
                               tiny ratio flags factors that may be
                               inaccurate; the refinement residual decides)   */
  int32_t krylov_iterations; /* FGMRES iterations summed over the sides,
                               refinement steps and filters of the call       */
} feast_nh_info;

/* inner_kind FEAST_NH_INNER_FGMRES (with precision FEAST_NH_PREC_FP32_IR):
 * the shifted systems are solved by restarted flexible GMRES in complex FP32
 * over every (node, column) system at once, right-preconditioned by
 * opts.precond, inside FP64 iterative refinement (each refinement step asks
 * FGMRES for a relative reduction of max(1e-5, inner_tol), at most
 * krylov_max iterations; the FP64 residual decides convergence). */

/* Fills *o with the defaults listed above. */
void feast_nh_default_opts(feast_nh_opts *o);

/* Creates a context for the pencil (A, B) on `contour` with subspace size m0
 * (1 <= m0 <= 128).  B == NULL means B = I.  `stream` is a cudaStream_t (NULL:
 * the legacy default stream).  Builds the transposed CSR of A and B for the
 * left (^H) products and the quadrature nodes; allocates all workspace.
 * Cite: Fig. alg:three inputs; Sec. 2.1 contour options. */
feast_nh_status feast_nh_init(feast_nh_ctx **ctx, const feast_nh_csr *A, const feast_nh_csr *B,
                              const feast_nh_contour *contour, int32_t m0,
                              const feast_nh_opts *opts, void *stream);

/* Contour integration, step 1 of Fig. alg:three (eq. qr, eq. ql): from the
 * n x m blocks Y, Yh computes Q and Qh (m <= m0).  Yh/Qh may be NULL for the
 * complex-symmetric problem, where Qh = conj(Q) (Sec. 2.4).  Factorises the
 * shifted matrices on first use and keeps the factors (Sec. 4.1 option).
 * Waits for the stream once, to read the largest relative residual
 * ||BY - (z_j B - A) X_j||_2 / ||BY||_2 of the shifted solves: above
 * opts.inner_tol it returns FEAST_NH_EINNER (Q, Qh then hold the filter of the
 * last iterates). */
feast_nh_status feast_nh_filter(feast_nh_ctx *ctx, const void *Y, const void *Yh, void *Q, void *Qh,
                                int32_t m);

/* Steps 2-4 of Fig. alg:three on n x m blocks Q, Qh: B_Q, spurious test
 * against the previous call's Ritz values, eigendecomposition of B_Q,
 * resize (eq. resize), B-bi-orthonormal U, Uh (eq. uu), reduced problem,
 * Ritz values `lambda` (device, m complex) and Ritz vectors Y, Yh (n x m_new,
 * row-major, leading dimension m_new).  Writes the new size to *m_new and,
 * if info != NULL, m_r/m_s/max_res of the convergence test (step 5). */
feast_nh_status feast_nh_rr(feast_nh_ctx *ctx, const void *Q, const void *Qh, int32_t m, double *lambda,
                            void *Y, void *Yh, int32_t *m_new, feast_nh_info *info);

/* The whole method (Fig. alg:three steps 0-5) from start blocks Y0, Yh0
 * (n x m0; Yh0 ignored for the complex-symmetric problem).  On return the
 * first *m_found columns of X, Xh (n x m0, leading dimension m0), entries of
 * lambda (m0 complex) and res (m0 doubles, eq. res) are the converged
 * eigenpairs inside C, normalised with ||x_i||_2 = 1 (largest entry real
 * positive) and x^_i^H B x_i = 1.  Returns FEAST_NH_ENOCONV after
 * opts.max_iter outer iterations, or FEAST_NH_EINNER instead when some
 * filter's shifted solves also stopped above their tolerance
 * (info->inner_fail counts them; a converged solve returns FEAST_NH_OK and
 * still reports the count). */
feast_nh_status feast_nh_solve(feast_nh_ctx *ctx, const void *Y0, const void *Yh0, double *lambda,
                               void *X, void *Xh, double *res, int32_t *m_found, feast_nh_info *info);

/* Attaches a trained network (feast_nh_net_*) as the right preconditioner of
 * the FGMRES inner solver (opts.precond == FEAST_NH_PRECOND_LEARNED).  The
 * operator must live on an N x N grid with n = N^2 (row i = y N + x, the
 * network's image layout).  Input channels per system (node j, column c):
 * Re v / rms(v), Im v / rms(v), kappa Re z_j, kappa Im z_j (conjugated for
 * the ^H side), then the nfeat <= 28 constant features (host floats); the
 * output channels 0, 1 scaled back by rms(v) are the preconditioned vector.
 * The context does not own the network; it must outlive the context's
 * filters. */
struct feast_nh_net;
/* Training pairs for the network from the method's own exact solves: with
 * ctx's banded direct solver (refined to opts.inner_tol), X_j = (z_j B -
 * A)^{-1} R for the n x m block R (device, complex double); for every system
 * s = j*m + c, Xin[s] (N x N x 32 floats, device) is column c of R packed as
 * the preconditioner packs its input (r / rms(r), kappa, features as in
 * feast_nh_set_network) and T[s] (N x N x 2 floats, device) is X_j[:, c] /
 * rms(R[:, c]), the exact correction of that normalised input.  Returns
 * FEAST_NH_EINNER if the solves missed inner_tol. */
feast_nh_status feast_nh_learned_pairs(feast_nh_ctx *ctx, const void *R, int32_t m, int32_t N, float kappa,
                                      const float *features, int32_t nfeat, float *Xin, float *T);
/* Operator-norm training loss of network outputs `out` (m*ne images, N x N x
 * 32 floats, device, channels 0 and 1 the complex correction) against the
 * exact corrections T (as from feast_nh_learned_pairs): for system s = j*m+c
 *     y_s = (z_j I - A)(out_s - T_s)       (side 1: (conj z_j I - A^H)),
 * loss = sum |y|^2 / (ne m n) (host), and d loss / d out into gout (device,
 * same shape as out, channels 2..31 zero).  Since (z_j I - A) T_s is the
 * input residual, this is the residual left by the network's correction:
 * it weighs errors by the operator, not by their size. */
feast_nh_status feast_nh_operator_loss(feast_nh_ctx *ctx, const float *out, const float *T, int32_t m, int32_t N,
                                      int32_t side, float *gout, double *loss);
feast_nh_status feast_nh_set_network(feast_nh_ctx *ctx, struct feast_nh_net *net, int32_t N, float kappa,
                                     const float *features, int32_t nfeat);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t feast_nh_kernel_launches(void);

/* Frees everything the context owns (not the caller's CSR arrays). */
void feast_nh_destroy(feast_nh_ctx *ctx);

/* Static description of a status code. */
const char *feast_nh_strerror(feast_nh_status s);

/* Message of the last failing call on ctx ("" if none). */
const char *feast_nh_last_error(const feast_nh_ctx *ctx);

/* Quadrature nodes and weights of a contour (host, 2*ne doubles each),
 * exactly those the filter uses (Sec. 2.3 trapezoidal rule). */
feast_nh_status feast_nh_nodes(const feast_nh_contour *contour, double *z, double *w);

/* Multi-shift sparse product used as the inner residual, exposed for
 * measurement: for every node j and column c,
 *   R_j = B Y - (z_j B - A) X_j       and  Q = sum_j w_j X_j  (if Q != NULL)
 * with X (ne blocks of n x m, node-major, device complex double), Y (n x m),
 * R (ne blocks, device).  Arithmetic in FP64; R is stored as complex double,
 * or as complex float (interleaved) when r_single != 0, the form the refined
 * single-precision solves read.  One pass over A and B (eq. qr). */
feast_nh_status feast_nh_multishift_residual(feast_nh_ctx *ctx, const void *X, const void *BY, void *R,
                                             void *Q, int32_t m, int32_t r_single);

/* The single-precision multi-shift operator of the Krylov sweeps (eq. qr /
 * eq. ql operators for every node at once): side 0: V_j = (z_j B - A) P_j,
 * side 1: V_j = (conj(z_j) B^H - A^H) P_j, for every node j and column c in
 * one pass over the CSR arrays.  P, V: ne node-major blocks of n x m
 * row-major complex FLOAT (interleaved), device, owned by the caller;
 * FP32 arithmetic.  Asynchronous on ctx's stream. */
feast_nh_status feast_nh_multishift_spmm(feast_nh_ctx *ctx, const void *P, void *V, int32_t m, int32_t side);

/* Eigen-decomposition of an m x m complex matrix M (device, row-major,
 * 1 <= m <= 128) by the library's small dense eigensolver, the one used for
 * B_Q = V Gamma V^^H (eq. bdiag, Sec. 2.5) and the reduced problem of step
 * 4.b: lambda (m complex) and right eigenvectors V (m x m, row-major, column
 * k for lambda_k), on ctx's stream with ctx's workspace.  Exposed so that the
 * eigensolver can be tested on its own.  Waits for the stream; a QR sweep
 * that does not converge returns FEAST_NH_ECUDA. */
feast_nh_status feast_nh_small_eig(feast_nh_ctx *ctx, const void *M, int32_t m, void *lambda, void *V);

/* G = X^H Y for device blocks X (n x mx) and Y (n x my), n = the context's
 * size, row-major complex double with leading dimensions mx and my;
 * G: mx x my, row-major (1 <= mx, my <= 128).  These are the projections of
 * steps 2.a and 4.a of Fig. alg:three (B_Q = Q^H B Q, A_U = Uh^H A U,
 * B_U = Uh^H B U).  method FEAST_NH_PROJ_TENSOR: every column is scaled by
 * the power of two of its largest component, each value becomes a 55-bit
 * fixed-point integer in eight signed 7-bit digits (exact in BF16), the 36
 * digit-pair products of significance >= 2^-49 are summed exactly on the
 * tensor cores (FP32 accumulators kept below 2^22) and in 64-bit integers,
 * and the sum is rounded once to FP64: |error| <= about 2^-52 max|x| max|y|
 * per term, and the result does not depend on the order of summation.
 * FEAST_NH_PROJ_FP64: FP64 on the CUDA cores.  On ctx's stream, with ctx's
 * workspace; waits for the stream.  Exposed so that the products can be
 * tested on their own; feast_nh_solve/feast_nh_rr use opts.projection. */
feast_nh_status feast_nh_gram(feast_nh_ctx *ctx, const void *X, const void *Y, int32_t mx, int32_t my, void *G,
                              int32_t method);

/* Z = X S for device blocks X (n x mx, leading dimension mx) and S (mx x mz,
 * leading dimension mz), Z: n x mz (leading dimension mz); row-major complex
 * double, 1 <= mx, mz <= 128: the block updates U = Q V Gamma^{-1/2}
 * (eq. uu) and Y = U W (step 4.d).  Methods as for feast_nh_gram, with the
 * scaling per row of X and per column of S.  Waits for the stream. */
feast_nh_status feast_nh_block_product(feast_nh_ctx *ctx, const void *X, const void *S, int32_t mx, int32_t mz,
                                       void *Z, int32_t method);

/* Device workspace of contexts and batches comes from one stream-ordered
 * memory pool per device, owned by the library (allocated in stream order on
 * the context's stream at init, returned in stream order at destroy).  The
 * pool keeps returned memory reserved, so a following init reuses it without
 * cudaMalloc / cudaFree; this call gives the reserved, unused memory back to
 * the driver (for example before other code needs the device memory).
 * Memory of live contexts is not affected.  Returns FEAST_NH_ECUDA if a trim
 * fails. */
feast_nh_status feast_nh_release_memory(void);

/* Device error-word bits, as reported through the status codes. */
enum { FEAST_NH_DEVERR_ZERO_PIVOT = 1, FEAST_NH_DEVERR_QR_NOCONV = 2, FEAST_NH_DEVERR_TIMEOUT = 16 };

/* Fault injection for tests, on the host: the next contour integration
 * (feast_nh_filter, or the first filter of feast_nh_solve) ORs `bits` into
 * the context's device error word after its kernels, so that the host's
 * mapping of that word to a status (FEAST_NH_ETIMEOUT for
 * FEAST_NH_DEVERR_TIMEOUT, ...) can be exercised without making a device
 * wait run out or a kernel fault.  One-shot. */
feast_nh_status feast_nh_inject_device_error(feast_nh_ctx *ctx, uint32_t bits);

/* The multi-shift residual above for callers that cannot allocate device
 * memory (an application that owns all device memory through its own pool or
 * budget, a latency-bound loop that cannot take the synchronisation of
 * cudaMalloc/cudaFree, an embedding whose memory footprint is fixed at
 * start-up).  The paper has no counterpart: this is an interface variant.
 *
 * Computes, with no context and no allocation, for every node j of `contour`
 * and column c:  R_j = BY - (z_j B - A) X_j,  Q = sum_j w_j X_j (if Q != NULL)
 * and relres[j*m + c] = ||R_jc||_2 / ||BY_c||_2.  A, B: device CSR as for
 * feast_nh_init (B == NULL: identity).  X, R: ne node-major blocks of n x m;
 * BY, Q: n x m; all row-major complex double in device memory, owned by the
 * caller; relres: ne*m device doubles.  Enqueued on `stream` (cudaStream_t).
 *
 * Scratch: a file-scope device array of 4.6 MiB (quadrature nodes, column
 * norms, partial sums of at most 256 CTAs) that every GPU loading the library
 * holds until exit.  Limits: 1 <= m <= 128, 1 <= ne <= 64, ne*m <= 2048;
 * larger sizes, NULL blocks or bad CSR descriptors return FEAST_NH_EINVAL
 * before any device work.  Runs on the CURRENT device: X, BY, R, Q, relres and
 * the CSR arrays must live there.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current)
 * and caches it; make that first call before any stream capture.  The
 * quadrature nodes are formed on the device by a kernel from the contour's
 * parameters (custom nodes are passed by value), so no host buffer is read
 * after the call returns.  All calls share the array: calls that overlap on
 * the GPU (other streams, other threads) race, so serialise them.  Every
 * scratch entry a call reads is written earlier in the same call, so nothing
 * carries over between calls.  A CUDA error left pending by earlier work of
 * the caller is reported as FEAST_NH_ECUDA before anything is enqueued. */
feast_nh_status feast_nh_multishift_residual_noalloc(const feast_nh_csr *A, const feast_nh_csr *B,
                                                     const feast_nh_contour *contour, const void *X,
                                                     const void *BY, void *R, void *Q, double *relres,
                                                     int32_t m, void *stream);

/* ------------------------------------------------------------------------
 * Many independent problems in one solve (the independence of contours and
 * of quadrature nodes, Sec. 4.1).  Problem p is the standard problem
 * (B = I) of its own CSR matrix A[p] (device, 0-based LOCAL column indices,
 * order n_p >= m0) on its own contour contours[p] (kinds 0, 1 or 2; the same
 * ne <= 16 for all).  The contour integration of every problem, node and
 * column runs in ONE persistent cooperative launch: shifted systems solved
 * by Jacobi-preconditioned BiCGStab inside iterative refinement (opts.
 * precision FP32_IR: single-precision Krylov sweeps, FP64 residuals and
 * updates; FP64: all in double), Q = sum_j w_j X_j per problem.  The
 * Rayleigh-Ritz step of each problem (Fig. alg:three steps 2-5) then runs
 * on that problem's own stream, all problems concurrently.  Converged
 * problems drop out; the others continue.  The launch shape (threads per
 * CTA, CTAs per SM, rows per tile) is chosen at init by timing candidates;
 * the launch sequence of one contour integration is captured once as a CUDA
 * graph (per inner tolerance) and replayed every outer iteration.
 *
 * Blocks are DEVICE complex double, rows of all problems concatenated in
 * problem order: problem p's rows start at off_p = n_0 + ... + n_{p-1}, and
 * its n_p x m0 row-major block starts at element off_p * m0 (so Y0 is a
 * C-contiguous (sum n_p, m0) array).  opts.inner_kind must be
 * FEAST_NH_INNER_BICGSTAB, opts.problem GENERAL; inner_tol, inner_max and
 * krylov_max bound the refinement and the Krylov iterations. */
typedef struct feast_nh_batch feast_nh_batch; /* opaque */

typedef struct {
  int32_t iterations;          /* outer iterations (the slowest problem)      */
  int32_t converged_problems;  /* problems whose test of step 5 passed        */
  int32_t inner_fail;          /* filters with a system above its tolerance   */
  int32_t krylov_iterations;   /* summed over filters, sides and refinements  */
  int32_t refine_steps;        /* summed over filters and sides               */
  int32_t threads, tile_rows, grid; /* launch shape the tuner chose          */
  double max_res;              /* largest eq. (res) residual returned         */
  double inner_res;            /* largest relative inner residual, last filter */
  double t_filter_ms, t_rr_ms, t_total_ms, t_autotune_ms;
  int32_t graph;               /* 1: the contour integration ran as a replayed
                                  CUDA graph of its launch sequence          */
} feast_nh_batch_info;

/* Creates the batch: per-problem transposed CSR (for the ^H solves),
 * quadrature nodes, workspace; runs the launch-shape tuner (a few short
 * launches on a fixed input).  Enqueued on `stream`; waits for it. */
feast_nh_status feast_nh_batch_init(feast_nh_batch **batch, int32_t nprob, const feast_nh_csr *A,
                                    const feast_nh_contour *contours, int32_t m0, const feast_nh_opts *opts,
                                    void *stream);

/* Solves every problem from start blocks Y0, Yh0 ((sum n_p) x m0).  Outputs
 * per problem p: m_found[p] (host) converged pairs inside its contour, first
 * in X, Xh (problem p's block at element off_p * m0, leading dimension m0),
 * lambda[p*m0 + k] (device, complex) and res[p*m0 + k] (device, eq. res),
 * normalised as for feast_nh_solve; iterations[p] (host, may be NULL) the
 * outer iterations problem p took.  Returns FEAST_NH_ENOCONV (or
 * FEAST_NH_EINNER if inner solves also missed) when some problem did not
 * converge within opts.max_iter. */
feast_nh_status feast_nh_batch_solve(feast_nh_batch *batch, const void *Y0, const void *Yh0, double *lambda,
                                     void *X, void *Xh, double *res, int32_t *m_found, int32_t *iterations,
                                     feast_nh_batch_info *info);

void feast_nh_batch_destroy(feast_nh_batch *batch);
const char *feast_nh_batch_last_error(const feast_nh_batch *batch);

/* ------------------------------------------------------------------------
 * Network of the learned preconditioner (the inner solves of step 1 accept
 * any solver, Sec. 3; this one is trained on the method's own exact solves):
 * `layers` 3x3 convolutions on an N x N grid, 32 channels, zero padding at
 * the grid boundary, ReLU between layers, none after the last:
 *     z_l = conv3x3(a_{l-1}; W_l) + b_l,  a_l = relu(z_l),  out = z_L.
 * BF16 weights and activations, FP32 accumulation on the tensor cores
 * (tcgen05), FP32 master parameters and Adam updates.  Images are DEVICE
 * float arrays, channel-last (image, y, x, channel), 32 channels.  Parameters
 * (HOST float arrays) are, per layer, W[tap][c_in][c_out] (tap = 3 dy + dx
 * for the neighbour offset (dy - 1, dx - 1); 9 * 32 * 32 values) followed by
 * b[32]: layers * 9248 floats in all.  All calls run on `stream` and wait for
 * it before returning. */
typedef struct feast_nh_net feast_nh_net; /* opaque */

/* Workspace for up to max_images images; parameters start at zero. */
feast_nh_status feast_nh_net_create(feast_nh_net **net, int32_t layers, int32_t N, int32_t max_images,
                                    void *stream);
feast_nh_status feast_nh_net_set_params(feast_nh_net *net, const float *params);
feast_nh_status feast_nh_net_get_params(feast_nh_net *net, float *params);
/* out = network(x), both nimg x N x N x 32 (device). */
feast_nh_status feast_nh_net_forward(feast_nh_net *net, const float *x, float *out, int32_t nimg);
/* One training step on the mean squared error of the first `cout` output
 * channels against `target` (nimg x N x N x cout, device):
 * loss = sum (out - target)^2 / (nimg N^2 cout).  Writes the loss (host) and,
 * if grad != NULL, the parameter gradient (device, layers * 9248 floats);
 * lr > 0 applies one Adam step (beta 0.9 / 0.999, eps 1e-8), lr = 0 none. */
feast_nh_status feast_nh_net_train_step(feast_nh_net *net, const float *x, const float *target, int32_t cout,
                                        int32_t nimg, float lr, double *loss, float *grad);
/* Backward pass from a given output gradient gout (nimg x N x N x 32,
 * device) through the activations of the last feast_nh_net_forward call on
 * the same images, parameter gradient into grad (device, may be NULL), one
 * Adam step if lr > 0. */
feast_nh_status feast_nh_net_backward(feast_nh_net *net, const float *gout, int32_t nimg, float lr, float *grad);
void feast_nh_net_destroy(feast_nh_net *net);
const char *feast_nh_net_last_error(const feast_nh_net *net);

#ifdef __cplusplus
}
#endif
#endif /* FEAST_NH_H */
