/*
 * seemps_gb300.h - C ABI of the GB300 (sm_103a) two-site variational sweep.
 *
 * The library implements the hot path of the MPS/TT method of "SeeMPS: A
 * Python-based Matrix Product State and Tensor Train Library": the two-site
 * sweep used for the eigenvalue search (DMRG, Sect. 3.1.1) and for the linear
 * solve U x = b (DMRG as a linear solver, Sect. 3.2.3).  Every step runs in
 * the library's own CUDA kernels.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All tensors are real float64, row-major (C order), in DEVICE memory,
 *   unless a parameter says "host".  The caller allocates and owns every
 *   tensor; the library never frees caller memory.
 * - MPS tensor A[alpha_{n-1}, s_n, alpha_n], shape (chi_l, d, chi_r): the
 *   storage order of Sect. 2.1.  MPO tensor W[b, j, i, f], shape
 *   (D_l, d, d, D_r) with j the output and i the input physical index: the
 *   storage order of Sect. 2.2.
 * - Quadratic-form environments (Sect. 2.5, the cached L and R of two-site
 *   DMRG): left L[a', b, a] of shape (chi, D, chi), contracting every site
 *   left of the active pair; right R[c', f, c] of shape (chi, D, chi),
 *   contracting every site right of it.  The first index is the bra (v), the
 *   last the ket (w) bond.  The boundary environments are the 1x1x1 tensor 1.
 * - Antilinear-form environments <v, w> (Sect. 2.5): F[a, a''] (left) and
 *   G[c, c''] (right), first index on v, second on w.
 * - Two-site vector a_n[a, s, t, c] = sum_m A_n[a, s, m] A_{n+1}[m, t, c],
 *   shape (chi_l, d, d, chi_r) (Sect. 2.5).
 * - Calls are asynchronous on the context's stream unless stated otherwise;
 *   results written to device pointers are ready once that stream reaches
 *   them.  Outputs may not alias inputs.
 * - Every call returns a seemps_status; nothing throws across the ABI.  On
 *   failure seemps_last_error() describes the first error.  Kernels never
 *   trap: a device-detected problem (a non-finite value, a bounded wait that
 *   ran out) is recorded in a device status word that
 *   seemps_device_status() reads.
 * - The context carves all temporary storage out of ONE workspace buffer
 *   that the caller allocates and passes to seemps_create();
 *   seemps_workspace_bytes() gives the size for given limits.  A call whose
 *   sizes exceed the workspace fails with SEEMPS_ERR_WORKSPACE and does
 *   nothing.
 *
 * Precision: SEEMPS_FP64 runs every contraction in FP64 on the CUDA cores.
 * SEEMPS_BF16X3 runs the dense contractions (environment update and the
 * effective operator) on the tcgen05 tensor cores with each FP64 operand
 * split as a = hi + lo (hi = bf16(a), lo = bf16(a - hi)) and
 * C = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulated in FP32; the result is
 * returned in FP64.  The environment updates split each operand into three
 * bf16 planes (a = hi + lo + lo2 to ~2^-24) and add the products hi lo2,
 * lo lo, lo2 hi (relative error ~2^-24): a sweep renews each environment
 * from the previous one, and two planes would let errors of ~1e-5 per
 * update accumulate over the chain.  Lanczos re-orthogonalisation, the tridiagonal
 * eigenproblem and the truncation sums stay FP64 in both modes; the Jacobi
 * rotations of the SVD run in FP32 in the bf16x3 sweep (their accuracy
 * matches that of the bf16x3 contractions) and in FP64 otherwise.
 * SEEMPS_FP64X2 (environment updates, effective operator, sweeps in eigen,
 * solve, simplify and apply modes) carries the quadratic-form environments
 * and the operator product in double-FP64: each value is an unevaluated sum
 * hi + lo of two doubles (about 106 significant bits), formed with
 * error-free products and sums on the FP64 units.  It is for operators whose
 * MPO adds channels of very different size, such as the QTT Laplacian of
 * Sect. 5.1 on 2^n points (channels of order 4^n cancelling to order 1),
 * where FP64 environments bound the relative error of a solve at about
 * eps 4^n / 40.  A double-FP64 tensor of n elements is a buffer of 2n
 * doubles: the n high parts, then the n low parts (the first half alone is
 * its FP64 rounding).  MPS tensors, vectors and the SVD stay FP64.
 */
#ifndef SEEMPS_GB300_H
#define SEEMPS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int seemps_status;
enum {
  SEEMPS_OK = 0,
  SEEMPS_ERR_INVALID = 1,        /* bad argument (null pointer, size <= 0, ...) */
  SEEMPS_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  SEEMPS_ERR_WORKSPACE = 3,      /* the workspace is too small for these sizes */
  SEEMPS_ERR_NOT_CONVERGED = 4,  /* an iteration hit its cap */
  SEEMPS_ERR_TIMEOUT = 5,        /* a bounded device wait ran out */
  SEEMPS_ERR_NUMERICAL = 6,      /* NaN / Inf met in a result */
  SEEMPS_ERR_UNSUPPORTED = 7     /* e.g. tensor-core path on a non-sm_103 device */
};

enum { SEEMPS_FP64 = 0, SEEMPS_BF16X3 = 1, SEEMPS_FP64X2 = 2 };
enum { SEEMPS_LEFT = 0, SEEMPS_RIGHT = 1 };
/* Truncation (Sect. 2.3): keep at most chi_max singular values and
 * - WEIGHT:   the fewest (r >= 1) whose discarded squared weight
 *             sum_{j>=r} s_j^2 is <= tol * sum_j s_j^2, both sums taken one
 *             term at a time from the smallest value upward (so equal s give
 *             equal r bit for bit);
 * - RELATIVE: those with s_j > tol * s_0 (the rule stated in Sect. 2.3). */
enum { SEEMPS_TRUNC_WEIGHT = 0, SEEMPS_TRUNC_RELATIVE = 1 };
/* Which side of the split receives the singular values: ABSORB_RIGHT for a
 * left-to-right step (A_n becomes a left isometry), ABSORB_LEFT for a
 * right-to-left step (A_{n+1} becomes a right isometry). */
enum { SEEMPS_ABSORB_RIGHT = 0, SEEMPS_ABSORB_LEFT = 1 };
enum { SEEMPS_PRECOND_NONE = 0, SEEMPS_PRECOND_JACOBI = 1, SEEMPS_PRECOND_MLP = 2 };
/* Sweep modes: two-site DMRG for the lowest eigenpair (Sect. 3.1.1); DMRG as a
 * linear solver U x = b (Sect. 3.2.3); variational compression of b to bond
 * dimension <= chi_max (Sect. 2.3, the minimiser of |x - b|^2; sums of MPS
 * are passed as their direct sum); two-site TDVP (Sect. 7.3, TDVP) for the
 * real generator L = -H, i.e. normalised imaginary-time evolution, one time
 * step tdvp_dt per sweep; the variational MPO-MPS product (Sect. 2.4.2, the
 * minimiser x of |x - W b|^2 at bond dimension <= chi_max, without forming
 * the enlarged product). */
enum { SEEMPS_MODE_EIG = 0, SEEMPS_MODE_SOLVE = 1, SEEMPS_MODE_SIMPLIFY = 2, SEEMPS_MODE_TDVP = 3,
       SEEMPS_MODE_APPLY = 4 };

typedef struct seemps_ctx seemps_ctx;

typedef struct {
  int chi_max;   /* maximum bond dimension kept */
  double tol;    /* tolerance of the truncation rule */
  int rule;      /* SEEMPS_TRUNC_WEIGHT or SEEMPS_TRUNC_RELATIVE */
} seemps_strategy;

/* Sizes of one two-site problem on the pair (n, n+1). */
typedef struct {
  int chi_l;  /* bond left of site n          */
  int chi_r;  /* bond right of site n+1       */
  int d;      /* physical dimension           */
  int D_l;    /* MPO bond left of site n      */
  int D_m;    /* MPO bond between n and n+1   */
  int D_r;    /* MPO bond right of site n+1   */
} seemps_pair_dims;

/* ---------------------------------------------------------------- context */

/* Workspace bytes needed for problems up to bond dimension chi_max, physical
 * dimension d, MPO bond D_max and Krylov dimension krylov_dim (and, for the
 * modes that read a second MPS b -- solve, simplify, apply -- b's bond
 * chib_max).  Host-only. */
seemps_status seemps_workspace_bytes(int chi_max, int d, int D_max, int krylov_dim,
                                     int chib_max, size_t* bytes_out);

/* Create a context on CUDA device `device`, issuing work on `stream` (a
 * cudaStream_t, 0 = the legacy default stream).  `workspace` is caller-owned
 * device memory of `workspace_bytes` bytes, 256-byte aligned, that must stay
 * valid until seemps_destroy().  Host-side allocation only (the context
 * struct and a pinned status word). */
seemps_status seemps_create(seemps_ctx** out, int device, void* stream, void* workspace,
                            size_t workspace_bytes);
seemps_status seemps_destroy(seemps_ctx* ctx);
seemps_status seemps_set_stream(seemps_ctx* ctx, void* stream);
/* Limit, in SM clocks, of the context's software waits on the device: the
 * grid barriers and block hand-offs of the cooperative Jacobi SVD kernels.
 * A block that waits longer gives up, records SEEMPS_ERR_TIMEOUT in the
 * status word (seemps_device_status) and returns; the call's results are
 * then invalid but the context stays usable.  Default (and the largest value
 * accepted; a negative value restores it): 2e9 clocks, about one second.  0
 * makes every wait that is not satisfied at once give up (used to test the
 * timeout path).  The tensor-core GEMM's mbarrier waits keep the default. */
seemps_status seemps_set_wait_limit(seemps_ctx* ctx, long long clocks);
/* Whether the bf16x3 effective operator applies the MPO mixing in the
 * epilogue of its first tensor-core GEMM (1) or in a kernel of its own
 * between the two GEMMs (0, the default: faster on GB300 at chi = 1024,
 * where the fused epilogue's mixing outlasts the next tile's MMAs).  Both give bit-identical results; the
 * fused form applies when d^2 (two sites) or d (one site) is a power of two
 * of at most 16, D_l d^2 and d^2 D_r are at most 32 and 128-row tiles of
 * whole D_l groups lose at most 1/8 of their rows (D_l in 1..6, 8, 16, 32);
 * other shapes always use the separate kernel. */
seemps_status seemps_set_fused_mixing(seemps_ctx* ctx, int enabled);
/* Text of the first error recorded on this context ("" if none). */
const char* seemps_last_error(const seemps_ctx* ctx);
/* Synchronises the stream and returns the device status word (SEEMPS_OK if
 * every kernel so far completed cleanly), then clears it. */
seemps_status seemps_device_status(seemps_ctx* ctx, int* status_out);
/* Number of kernels this context has launched so far (host counter). */
seemps_status seemps_launch_count(const seemps_ctx* ctx, long long* count_out);

/* Per-phase timing with CUDA events recorded on the context's stream (off by
 * default).  Phases: */
enum {
  SEEMPS_PHASE_MATVEC = 0,   /* one effective-operator apply */
  SEEMPS_PHASE_TC_GEMM = 1,  /* one tcgen05 GEMM launch (inside a matvec or env update) */
  SEEMPS_PHASE_LOCAL = 2,    /* one local solve (Lanczos or PCG, matvecs included) */
  SEEMPS_PHASE_SVD = 3,      /* one truncated SVD split */
  SEEMPS_PHASE_ENV = 4,      /* one environment update */
  SEEMPS_PHASE_JACOBI = 5,   /* the Jacobi kernel of one mixed-precision SVD (inside SVD) */
  SEEMPS_PHASE_QR = 6,       /* the QR preconditioning of one mixed-precision SVD (inside SVD) */
  SEEMPS_PHASE_COUNT = 8
};
seemps_status seemps_set_timing(seemps_ctx* ctx, int enabled);
/* Synchronises the stream, then returns the accumulated milliseconds and
 * the number of timed intervals of each phase (arrays of SEEMPS_PHASE_COUNT,
 * host memory); reset != 0 clears the accumulators. */
seemps_status seemps_get_timing(seemps_ctx* ctx, double* ms_out, long long* count_out, int reset);

/* ---------------------------------------------------------------- tile autotuner
 * The bf16x3 tensor-core GEMM has two tile shapes (128 x 128 and 128 x 256
 * outputs per CTA) whose results are bit-identical; which is faster depends
 * on the GEMM's shape.  seemps_autotune times both on the bf16x3 GEMMs of a
 * pair update at the sizes `dims` (effective operator, two-site tensor, the
 * split's second factor; the environment updates use the six-product GEMM,
 * which has one tile shape) and records the
 * faster per (device, M, N, padded K, output type) in a process-wide table
 * shared by all contexts; *tuned_out (host, may be NULL) receives the number
 * of shapes newly timed.  It synchronises the stream (do not call it during
 * stream capture) and draws its operands from the workspace (a shape that
 * does not fit stays untuned).  A context uses the table only after
 * seemps_set_autotune(ctx, 1); untuned shapes then, and every shape
 * otherwise, take a fixed rule (128 x 256 tiles from 1.5 waves of them on).
 * seemps_autotune_stats (host outputs, each may be NULL): lookups that found
 * a recorded shape, shapes this context timed, and entries in the table. */
seemps_status seemps_autotune(seemps_ctx* ctx, const seemps_pair_dims* dims, int* tuned_out);
seemps_status seemps_set_autotune(seemps_ctx* ctx, int enabled);
seemps_status seemps_autotune_stats(const seemps_ctx* ctx, long long* hits_out, long long* shapes_out,
                                    int* table_size_out);

/* ---------------------------------------------------------------- environments
 * Quadratic form (Sect. 2.5, Eqs. of the QuadraticForm environments):
 *  side = LEFT : E_out[c', f, c] = sum conj(A[a', s', c']) E_in[a', b, a] W[b, s', s, f] A[a, s, c]
 *                A has shape (chi_in, d, chi_out); W (D_in, d, d, D_out);
 *                E_in (chi_in, D_in, chi_in); E_out (chi_out, D_out, chi_out).
 *  side = RIGHT: E_out[a', b, a] = sum conj(A[a', s', c']) W[b, s', s, f] E_in[c', f, c] A[a, s, c]
 *                A has shape (chi_out, d, chi_in); W (D_out, d, d, D_in);
 *                E_in (chi_in, D_in, chi_in); E_out (chi_out, D_out, chi_out).
 * precision: SEEMPS_FP64, SEEMPS_BF16X3, or SEEMPS_FP64X2 (E_in and E_out
 * double-FP64: 2 chi_in^2 D_in and 2 chi_out^2 D_out doubles). */
seemps_status seemps_env_update(seemps_ctx* ctx, int side, int chi_in, int chi_out, int d,
                                int D_in, int D_out, const double* E_in, const double* A,
                                const double* W, double* E_out, int precision);

/* Environment of <x, W b> for two different MPS (Sect. 2.4.2, the variational
 * MPO-MPS product; the quadratic form above is the case X = B):
 *  side = LEFT : E_out[c', f, c] = sum conj(X[a', s', c']) E_in[a', b, a] W[b, s', s, f] B[a, s, c]
 *                X (chi_in_x, d, chi_out_x), B (chi_in_b, d, chi_out_b), W (D_in, d, d, D_out),
 *                E_in (chi_in_x, D_in, chi_in_b), E_out (chi_out_x, D_out, chi_out_b).
 *  side = RIGHT: E_out[a', b, a] = sum conj(X[a', s', c']) W[b, s', s, f] E_in[c', f, c] B[a, s, c]
 *                X (chi_out_x, d, chi_in_x), B (chi_out_b, d, chi_in_b), W (D_out, d, d, D_in),
 *                E_in (chi_in_x, D_in, chi_in_b), E_out (chi_out_x, D_out, chi_out_b).
 * precision: SEEMPS_FP64, SEEMPS_BF16X3 or SEEMPS_FP64X2 (E_in, E_out
 * double-FP64); errors as seemps_env_update. */
seemps_status seemps_env_update_braket(seemps_ctx* ctx, int side, int chi_in_x, int chi_in_b,
                                       int chi_out_x, int chi_out_b, int d, int D_in, int D_out,
                                       const double* E_in, const double* X, const double* B,
                                       const double* W, double* E_out, int precision);

/* Antilinear form <v, w> (Sect. 2.5), FP64:
 *  side = LEFT : F_out[c, c''] = sum conj(A[a, s, c]) F_in[a, a''] B[a'', s, c'']
 *                A (chi_in, d, chi_out), B (chib_in, d, chib_out), F_in (chi_in, chib_in).
 *  side = RIGHT: G_out[a, a''] = sum conj(A[a, s, c]) G_in[c, c''] B[a'', s, c'']
 *                A (chi_out, d, chi_in), B (chib_out, d, chib_in), G_in (chi_in, chib_in). */
seemps_status seemps_env_update_linear(seemps_ctx* ctx, int side, int chi_in, int chi_out,
                                       int chib_in, int chib_out, int d, const double* F_in,
                                       const double* A, const double* B, double* F_out);

/* ---------------------------------------------------------------- local operators */

/* a_n = A_n A_{n+1} (Sect. 2.5): A1 (chi_l, d, chi_m), A2 (chi_m, d, chi_r),
 * theta (chi_l, d, d, chi_r). FP64. */
seemps_status seemps_two_site(seemps_ctx* ctx, int chi_l, int chi_m, int chi_r, int d,
                              const double* A1, const double* A2, double* theta);

/* Effective operator of the pair (the H_n of Sect. 3.1.1):
 *  y[a', s', t', c'] = sum L[a', b, a] W1[b, s', s, e] W2[e, t', t, f] R[c', f, c] theta[a, s, t, c]
 * L (chi_l, D_l, chi_l), W1 (D_l, d, d, D_m), W2 (D_m, d, d, D_r),
 * R (chi_r, D_r, chi_r), theta and y (chi_l, d, d, chi_r).  With
 * SEEMPS_FP64X2, L and R are double-FP64 (hi parts, then lo parts) and the
 * product is accumulated in double-FP64 before y (FP64) is rounded once. */
seemps_status seemps_heff_apply(seemps_ctx* ctx, const seemps_pair_dims* dims, const double* L,
                                const double* W1, const double* W2, const double* R,
                                const double* theta, double* y, int precision);

/* The pair's MPO action between two MPS (Sect. 2.4.2, the local vector
 * (W b)_n of the variational MPO-MPS product):
 *  y[a', s', t', c'] = sum L[a', b, a] W1[b, s', s, e] W2[e, t', t, f] R[c', f, c] theta_b[a, s, t, c]
 * dims->chi_l, chi_r are x's bonds (y is (chi_l, d, d, chi_r)); chib_l, chib_r
 * are b's bonds (theta_b is (chib_l, d, d, chib_r)); L (chi_l, D_l, chib_l),
 * R (chi_r, D_r, chib_r), W1, W2 as in seemps_heff_apply.  y may not alias
 * theta_b. */
seemps_status seemps_heff_apply_braket(seemps_ctx* ctx, const seemps_pair_dims* dims, int chib_l,
                                       int chib_r, const double* L, const double* W1, const double* W2,
                                       const double* R, const double* theta_b, double* y, int precision);

/* diag(H_n)[a, s, t, c] = sum_{b,e,f} L[a,b,a] W1[b,s,s,e] W2[e,t,t,f] R[c,f,c]  (FP64),
 * the Jacobi preconditioner of the local solve. */
seemps_status seemps_heff_diagonal(seemps_ctx* ctx, const seemps_pair_dims* dims, const double* L,
                                   const double* W1, const double* W2, const double* R,
                                   double* diag);

/* b_n[a, s, t, c] = sum F[a, a''] B1[a'', s, e] B2[e, t, c''] G[c, c''] (Sect. 3.2.3, the
 * right-hand side of U_n a_n = b_n), FP64.  F (chi_l, chib_l), B1 (chib_l, d, chib_m),
 * B2 (chib_m, d, chib_r), G (chi_r, chib_r), b (chi_l, d, d, chi_r). */
seemps_status seemps_b_effective(seemps_ctx* ctx, int chi_l, int chi_r, int chib_l, int chib_m,
                                 int chib_r, int d, const double* F, const double* B1,
                                 const double* B2, const double* G, double* b);

/* The same FP64 effective-operator apply as seemps_heff_apply(SEEMPS_FP64),
 * for callers that cannot allocate device memory (their device memory is
 * owned by an allocator that will not give them a buffer, or they must not
 * trigger an allocation at all): it needs no context and no workspace.  The
 * paper has no counterpart; this is a deployment convenience.
 *  - Its intermediates live in one library-owned static device array of
 *    32 MiB, held by every GPU that loads the library until the process
 *    exits.  Sizes whose intermediates do not fit (about
 *    chi_l * chi_r * d^2 * (D_l + D_r) * 8 bytes) are rejected with
 *    SEEMPS_ERR_WORKSPACE before anything runs.
 *    Dimensions above chi = 2^20 or d, D = 2^10 are rejected with
 *    SEEMPS_ERR_INVALID (sizes are computed with overflow checks).
 *  - The first call in each CUDA context (the device's primary context or a
 *    driver-API context), with that context current, looks up the array's
 *    device address once and caches it under the context's process-unique
 *    id (a context recreated after cudaDeviceReset is looked up afresh);
 *    make that first call before any stream capture.
 *  - All calls share the array: calls whose kernels overlap on the GPU
 *    (other streams, other host threads) race.  Serialise them.
 *  - Runs on `stream` (a cudaStream_t, 0 = legacy default stream) of the
 *    current device; inputs and y as in seemps_heff_apply.
 *  - On failure a message is written to errbuf (may be NULL). */
seemps_status seemps_heff_apply_noalloc(const seemps_pair_dims* dims, const double* L,
                                        const double* W1, const double* W2, const double* R,
                                        const double* theta, double* y, void* stream,
                                        char* errbuf, size_t errbuf_len);

/* One-site effective operator (Sect. 7.3, TDVP; the one-site form of
 * Sect. 2.5's quadratic form):
 *   y[a', s', c'] = sum L[a', b, a] W[b, s', s, f] R[c', f, c] A[a, s, c]
 * dims: chi_l, chi_r, d, D_l, D_r as for a pair (D_m ignored); A and y are
 * (chi_l, d, chi_r); W is (D_l, d, d, D_r).  y may not alias A. */
seemps_status seemps_heff1_apply(seemps_ctx* ctx, const seemps_pair_dims* dims, const double* L,
                                 const double* W, const double* R, const double* A, double* y,
                                 int precision);

/* ---------------------------------------------------------------- local solvers */

/* exp(tau H) theta / |exp(tau H) theta| (Sect. 7.3, TDVP: the local steps with
 * the generator L = -H) in the Krylov space of theta: the Lanczos basis and
 * tridiagonal T of seemps_local_eig's recurrence, exp(tau T) e_1 from the
 * eigendecomposition of T (Jacobi), combined and normalised into theta.
 * sites = 2: H is the pair operator of W1, W2 (theta (chi_l, d, d, chi_r));
 * sites = 1: the one-site operator of W1 (theta (chi_l, d, chi_r), W2 may be
 * NULL).  alpha0_out (1 double, <theta, H theta>/<theta, theta>) and
 * iters_out (1 int) are DEVICE pointers (may be NULL). */
seemps_status seemps_local_expm(seemps_ctx* ctx, const seemps_pair_dims* dims, int sites, const double* L,
                                const double* W1, const double* W2, const double* R, double* theta_inout,
                                int krylov_dim, double breakdown_tol, double tau, int precision,
                                double* alpha0_out, int* iters_out);

/* Lowest eigenpair of H_n (Sect. 3.1.1: the local problem H_n a = E a with
 * the centre on the pair, so N_n = 1) by Lanczos from theta:
 * v_0 = theta/|theta|; k = krylov_dim steps with full re-orthogonalisation
 * (classical Gram-Schmidt, applied twice, FP64); stop early when
 * beta_j <= breakdown_tol * max(1, |alpha_0|).  theta_inout receives the
 * normalised Ritz vector of the lowest eigenvalue of the tridiagonal matrix.
 * energy_out (1 double) and iters_out (1 int) are DEVICE pointers. */
seemps_status seemps_local_eig(seemps_ctx* ctx, const seemps_pair_dims* dims, const double* L,
                               const double* W1, const double* W2, const double* R,
                               double* theta_inout, int krylov_dim, double breakdown_tol,
                               int precision, double* energy_out, int* iters_out);

/* Learned diagonal-plus-low-rank preconditioner for the local PCG solve.
 * The paper leaves the local solver open (Sect. 3.2.3: a standard iterative
 * method); this learned preconditioner is an addition.  For the entry j = (a, s, t, c) of
 * the local system on the pair (i, i+1) of an N-site chain the features
 *   (log10(diag_j)/10, i/N, (i+1)/N, log10|L[a,:,a]|/10, log10|R[c,:,c]|/10,
 *    s/(d-1), t/(d-1))
 * go through a 7 -> 64 -> 64 -> 5 tanh network (FP32) whose outputs o give
 *   p_j = softplus(o_0j)/diag_j,  U_jk = o_{1+k,j}/sqrt(n)  (k < 4),
 * and P = diag(p) + U U^T (symmetric positive definite).  Parameters are one
 * flat float32 DEVICE vector owned by the caller, ordered W1 (64x7), b1,
 * W2 (64x64), b2, W3 (5x64), b3 (weights row-major, out x in). */
typedef struct seemps_mlp seemps_mlp;

/* Number of float parameters for the given hidden width (only 64). Host-only. */
seemps_status seemps_mlp_param_count(int hidden, int* count);
/* Wrap caller-owned device parameters (not copied; must outlive the handle). */
seemps_status seemps_mlp_create(seemps_mlp** out, int hidden, float* params);
seemps_status seemps_mlp_destroy(seemps_mlp* mlp);
/* Position used for the i/N features by seemps_local_pcg (the sweep sets it
 * itself for every pair). */
seemps_status seemps_mlp_set_site(seemps_mlp* mlp, int site, int n_sites);
/* p (n doubles) and U (n x 4 doubles, row-major) of the local system. */
seemps_status seemps_mlp_forward(seemps_ctx* ctx, const seemps_mlp* mlp, const seemps_pair_dims* dims,
                                 const double* L, const double* W1, const double* W2,
                                 const double* R, double* p_out, double* U_out);
/* Loss |x* - P b|_A^2 / (x*^T b) of one system (A = H_n, FP64 apply) and its
 * gradient with respect to the parameters; both are ADDED to *loss_accum
 * (device double, may be NULL) and grad_accum (device floats). */
seemps_status seemps_mlp_loss_grad(seemps_ctx* ctx, const seemps_mlp* mlp,
                                   const seemps_pair_dims* dims, const double* L,
                                   const double* W1, const double* W2, const double* R,
                                   const double* b, const double* xstar, float* grad_accum,
                                   double* loss_accum);
/* One Adam step (Kingma & Ba, bias-corrected, step t >= 1) on the
 * parameters with gradient grad * grad_scale; m and v are caller-owned
 * device moment vectors. */
seemps_status seemps_mlp_adam(seemps_ctx* ctx, seemps_mlp* mlp, const float* grad, float* m,
                              float* v, int t, float lr, float beta1, float beta2, float eps,
                              float grad_scale);

/* Training set of local systems for seemps_mlp_train: host arrays of length
 * n_systems with the sizes, the device pointers of each system's operands
 * (L, W1, W2, R as in seemps_heff_apply, FP64), its right-hand side b and its
 * exact solution xstar, and the pair position (site, n_sites) of its
 * features. */
typedef struct {
  int n_systems;
  const seemps_pair_dims* dims;
  const double* const* L;
  const double* const* W1;
  const double* const* W2;
  const double* const* R;
  const double* const* b;
  const double* const* xstar;
  const int* site;
  const int* n_sites;
} seemps_mlp_dataset;

typedef struct {
  int steps;    /* Adam steps */
  int batch;    /* systems per step, taken cyclically (<= 0: all) */
  float lr, beta1, beta2, eps;
} seemps_mlp_train_params;

/* Train the network on its own GPU kernels: per step the mean of
 * seemps_mlp_loss_grad over the mini-batch, then seemps_mlp_adam.  grad, m
 * and v are caller-owned device float buffers of the parameter count (m, v
 * carry the Adam moments between calls); *t_inout (host) is the Adam step
 * counter, advanced by `steps`.  loss_history (host, `steps` doubles, may be
 * NULL) receives each step's mean loss and then costs one stream
 * synchronisation per step. */
seemps_status seemps_mlp_train(seemps_ctx* ctx, seemps_mlp* mlp, const seemps_mlp_dataset* data,
                               const seemps_mlp_train_params* params, float* grad, float* m, float* v,
                               int* t_inout, double* loss_history);

/* Solve H_n x = b (Sect. 3.2.3, Eq. of the projected system U_n a_n - b_n = 0)
 * by preconditioned conjugate gradients from x_inout, stopping when
 * |r| <= rtol |b| or after maxiter steps.  precond: NONE, JACOBI (diag H_n)
 * or MLP (needs mlp != NULL).  resid_out (relative residual, 1 double) and
 * iters_out (1 int) are DEVICE pointers.  Returns SEEMPS_OK even when the cap
 * is hit; the residual tells. */
seemps_status seemps_local_pcg(seemps_ctx* ctx, const seemps_pair_dims* dims, const double* L,
                               const double* W1, const double* W2, const double* R,
                               const double* b, double* x_inout, int precond,
                               const seemps_mlp* mlp, double rtol, int maxiter, int precision,
                               double* resid_out, int* iters_out);

/* ---------------------------------------------------------------- split */

/* Truncated SVD split of theta viewed as the m x n matrix M (Sect. 2.3;
 * m = chi_l d, n = d chi_r).  M = U S V^T by one-sided Jacobi in FP64; the
 * singular values are sorted descending (ties by column index), the rank r
 * follows `st`, and
 *   ABSORB_RIGHT: A_left = U_r (m x r), A_right = S~ V_r^T (r x n)
 *   ABSORB_LEFT : A_left = U_r S~ (m x r), A_right = V_r^T (r x n)
 * with S~ = S_r / |S_r| if normalize, else S_r.  A_left is written with row
 * stride r and A_right with row stride n.  S receives all min(m, n) singular
 * values (descending).  rank_out (1 int) and discarded_out (1 double: the
 * discarded fraction sum_{j>=r} s_j^2 / sum_j s_j^2) are DEVICE pointers.
 * max_sweeps bounds the Jacobi sweeps (0 = default 40).  precision:
 * SEEMPS_FP64 rotates in FP64; SEEMPS_BF16X3 (the mixed sweep) rotates in
 * FP32, with the norms, the truncation sums and the outputs in FP64.  For
 * large mixed problems (p = min(m, n) >= 64) a block sweep that rotates at
 * most p (p - 1) / 128 pairs hands over to a cleanup phase that checks only the
 * pairs of the columns it rotated and rotates disjoint violating pairs until
 * none is left (the same stopping rule: every pair within the threshold);
 * if it cannot finish, block sweeps continue from its columns. */
seemps_status seemps_svd_truncate(seemps_ctx* ctx, int m, int n, const double* theta,
                                  const seemps_strategy* st, int absorb, int normalize,
                                  double* A_left, double* A_right, double* S, int* rank_out,
                                  double* discarded_out, int max_sweeps, int precision);

/* The truncation rank alone, for s (device, n values, descending): the rule
 * of seemps_strategy evaluated by one thread in the fixed order stated
 * above.  rank_out is a DEVICE pointer. */
seemps_status seemps_truncation_rank(seemps_ctx* ctx, int n, const double* s,
                                     const seemps_strategy* st, int* rank_out);

/* Counters of the large-problem Jacobi SVD kernel (the bf16x3 sweep's path)
 * since the context was created or last reset: calls, Jacobi sweeps, pair
 * visits (column pairs whose dot product was formed; pairs skipped because
 * neither column changed since their previous visit are not counted) and
 * algorithmic FP32 operations (2 per element of a visited pair for its dot
 * product, 6 per element of a rotated pair).  Host-only; any pointer may be
 * NULL. */
seemps_status seemps_svd_stats(seemps_ctx* ctx, long long* calls, long long* sweeps,
                               long long* pair_visits, double* flops, int reset);

/* Per-sweep counters of the most recent large-problem Jacobi SVD on this
 * context: rotations[i] and visits[i] for sweep i < *n_sweeps (the last
 * sweep, without rotations, included).  At most `cap` entries are written
 * to each host array; *n_sweeps receives the full count (0 before the first
 * call).  Host-only diagnostics; no counterpart in the paper. */
seemps_status seemps_svd_sweep_counts(seemps_ctx* ctx, int* rotations, int* visits, int cap,
                                      int* n_sweeps);

/* Counters of the cleanup phase of the large-problem Jacobi SVD since the
 * context was created or last reset: splits that used it, its rounds
 * (checks of the changed columns' pairs, each followed by one set of
 * disjoint rotations) and fallbacks to block sweeps (a round found more than
 * 4096 violating pairs or 48 rounds did not finish).  Host-only; any
 * pointer may be NULL. */
seemps_status seemps_svd_cleanup_stats(seemps_ctx* ctx, long long* calls, long long* rounds,
                                       long long* fallbacks, int reset);

/* ---------------------------------------------------------------- sweep */

/* One chain.  Host arrays of device pointers; every A[i] has room for
 * chi_max * d * chi_max doubles, every environment for chi_max * D_max *
 * chi_max (quadratic), chi_max * D_max * chib_max (apply mode: Lenv/Renv
 * are the environments of <x, W b>, shape (chi, D, chib)) or chi_max *
 * chib_max (linear) doubles; sweeps in SEEMPS_FP64X2 need twice that room
 * in Lenv / Renv (double-FP64 environments). */
typedef struct {
  int n_sites;
  int d;
  /* MPO and quadratic-form environments: eigen, solve, TDVP and apply modes
   * (may be NULL in simplify mode) */
  const int* D;              /* host, n_sites + 1 MPO bond dims (D[0] = D[N] = 1) */
  const double* const* W;    /* host array of n_sites device MPO tensors */
  double** A;                /* host array of n_sites device MPS tensors (in/out) */
  int* chi;                  /* host, n_sites + 1 MPS bond dims (in/out) */
  double** Lenv;             /* host array of n_sites + 1 device buffers */
  double** Renv;             /* host array of n_sites + 1 device buffers */
  /* b: solve, simplify and apply modes (may be NULL in eigen and TDVP modes);
   * the antilinear-form environments: solve and simplify modes only */
  const double* const* B;    /* host array of n_sites device MPS tensors of b */
  const int* chib;           /* host, n_sites + 1 bond dims of b */
  double** Fenv;             /* host array of n_sites + 1 device buffers */
  double** Genv;             /* host array of n_sites + 1 device buffers */
} seemps_chain;

typedef struct {
  int mode;              /* SEEMPS_MODE_* */
  int n_sweeps;          /* sweeps in `precision` */
  int refine_sweeps;     /* extra sweeps in FP64 after them (environments rebuilt in FP64) */
  int precision;         /* SEEMPS_FP64, SEEMPS_BF16X3, or SEEMPS_FP64X2 (not TDVP; the
                            Lenv / Renv buffers then hold twice the doubles) */
  int krylov_dim;        /* Lanczos steps per pair (eigen mode) */
  double breakdown_tol;  /* Lanczos breakdown tolerance */
  seemps_strategy strategy;
  int canonicalize;      /* 1: bring the input MPS to right-canonical form first */
  double pcg_rtol;       /* solve mode */
  int pcg_maxiter;       /* solve mode */
  int precond;           /* solve mode: SEEMPS_PRECOND_* */
  const seemps_mlp* mlp; /* solve mode, SEEMPS_PRECOND_MLP */
  double tdvp_dt;        /* TDVP mode: the time step of one sweep (> 0) */
} seemps_sweep_params;

typedef struct {
  double energy;              /* eigen mode: energy of the last local solve */
  double max_discarded;       /* largest discarded fraction of any split */
  double error_bound;         /* sum of the discarded fractions (the accumulated bound of Sect. 2.3) */
  long long local_iters;      /* total Lanczos steps or PCG iterations */
  double seconds;             /* wall time of the call */
  int half_sweeps;            /* number of half sweeps done */
  double* half_sweep_energy;  /* host, optional (NULL): one value per half sweep */
  int* half_sweep_max_rank;   /* host, optional (NULL) */
} seemps_sweep_report;

/* Full sweeps over one chain (Sect. 2.5's sweep: pairs 0..N-2 left to right,
 * then N-2..0 right to left).  Eigen mode runs two-site DMRG (Sect. 3.1.1),
 * solve mode DMRG as a linear solver (Sect. 3.2.3), simplify, TDVP and apply
 * modes as described at SEEMPS_MODE_*.  On entry the chain's
 * MPS is either right-canonical with the centre on site 0 (canonicalize = 0)
 * or any MPS (canonicalize = 1).  On return the centre is on site 0 again.
 * Synchronises the stream (reads ranks and energies on the host). */
seemps_status seemps_sweep(seemps_ctx* ctx, seemps_chain* chain, const seemps_sweep_params* p,
                           seemps_sweep_report* report);

/* Sweeps over many independent chains at once (the batched workload of
 * many chains of uneven length and bond dimension).  Chain k runs
 * seemps_sweep(ctxs[k], chains[k], params[k], &reports[k]); every chain
 * needs its own context (its own stream and workspace: the same context
 * twice is rejected with SEEMPS_ERR_INVALID).  A pool of up to max_threads
 * host threads (0 = 16) drives the chains concurrently so that their kernels
 * overlap on the GPU.  statuses (host, n_chains) receives each chain's
 * status; reports (host, n_chains) may be NULL.  Blocks until every chain
 * is done; returns the first non-OK status, if any. */
seemps_status seemps_sweep_batch(seemps_ctx* const* ctxs, seemps_chain* const* chains,
                                 const seemps_sweep_params* const* params, int n_chains,
                                 int max_threads, seemps_sweep_report* reports,
                                 seemps_status* statuses);

/* A contiguous run of `count` pair updates of a sweep, starting at the pair
 * (first, first+1) and moving right (direction = +1: pairs first,
 * first+1, ...) or left (direction = -1: pairs first, first-1, ...).  The
 * chain must already be in mixed canonical form with the centre on the
 * first pair's sites and valid environments on both sides (as left by
 * seemps_sweep or by a previous range).  p->n_sweeps and p->refine_sweeps
 * are ignored; the contractions use p->precision.  The report's
 * half_sweep_* arrays are not written. */
seemps_status seemps_sweep_range(seemps_ctx* ctx, seemps_chain* chain,
                                 const seemps_sweep_params* p, int first, int count,
                                 int direction, seemps_sweep_report* report);

/* Rebuild the right environments R_N .. R_{first+2} (and G for solve mode)
 * from the chain's current MPS, in `precision`; the left ones L_0 .. L_first
 * likewise.  Used to prepare a chain for seemps_sweep_range. */
seemps_status seemps_build_environments(seemps_ctx* ctx, seemps_chain* chain, int mode,
                                        int first, int precision);

/* ---------------------------------------------------------------- global solver */

/* Conjugate gradients on MPS for U x = b with U a symmetric positive definite
 * MPO (Sect. 3.2.1, the CGS listing of Fig. cgs), every vector an MPS of bond
 * dimension <= strategy.chi_max:
 *   x = simplify(guess); r = b - U x; p = r; then per step
 *   alpha = |r|^2 / <p, U p>, x = simplify(x + alpha p), r = b - U x,
 *   beta = (|r_new| / |r_old|)^2, p = simplify(r + beta p),
 * until |r| < rtol |b|, |r| = 0 or maxiter steps.  Sums are joined MPS (Sect. 2.4.1)
 * compressed by the simplify sweep, U x the variational MPO-MPS product
 * sweep, each with n_sweeps sweeps started from the previous value of the
 * same MPS; |r| is the norm of the compressed residual, and |r|, <p, U p>
 * and |b| are FP64 contractions of the forms' environments (Sect. 2.5).
 * Where the printed listing departs from the standard recurrence the paper
 * cites (the sign of the step, the square in beta), the standard one is
 * taken.  Synchronises the stream once per step (two scalars). */
typedef struct {
  int n_sites;
  int d;
  const int* D;              /* host, n_sites + 1 MPO bonds (D[0] = D[N] = 1) */
  const double* const* W;    /* host array of n_sites device MPO tensors (D_l, d, d, D_r) */
  const int* chib;           /* host, n_sites + 1 bonds of b */
  const double* const* B;    /* host array of n_sites device tensors of b */
  int* chix;                 /* host, n_sites + 1 bonds of x: in the guess, out the solution */
  double** X;                /* host array of n_sites device buffers of x (in: guess, out:
                                solution), each with room for chi_max * d * chi_max doubles */
  void* work;                /* device arena of seemps_cgs_work_bytes() bytes (caller-owned) */
  size_t work_bytes;
} seemps_cgs_problem;

typedef struct {
  seemps_strategy strategy;  /* truncation of every compression (chi_max, tol, rule) */
  int n_sweeps;              /* sweeps per compression (>= 1) */
  int precision;             /* of the sweeps: SEEMPS_FP64 or SEEMPS_BF16X3 */
  int maxiter;               /* conjugate-gradient steps at most (>= 0) */
  double rtol;               /* stop when |r| < rtol |b| */
} seemps_cgs_params;

typedef struct {
  int iterations;            /* steps taken */
  double residual;           /* |r| at exit */
  double norm_b;             /* |b| */
  double seconds;            /* host wall time */
  double* residual_history;  /* host, optional (NULL): |r| after 0..iterations steps
                                (room for maxiter + 1 values) */
} seemps_cgs_report;

/* Bytes of the work arena for n_sites sites, physical dimension d, MPO bond
 * D_max, bond limit chi_max and b's bond chib_max: three work MPS (U x, r,
 * p), one joined MPS of bond chi_max + max(chi_max, chib_max), and the
 * sweeps' environments.  Host-only. */
seemps_status seemps_cgs_work_bytes(int n_sites, int d, int D_max, int chi_max, int chib_max,
                                    size_t* bytes_out);

/* Runs the solver on ctx's stream.  The context must have been sized with
 * chib_max >= chi_max + max(chi_max, chib) and D_max >= the MPO's bonds (the
 * sweeps it runs read joined MPS of that bond).  Errors: SEEMPS_ERR_INVALID
 * for a bad argument, a guess bond outside [1, chi_max], a too small arena,
 * or <p, U p> <= 0 (U not positive definite); the sweeps' own errors pass
 * through. */
seemps_status seemps_cgs_solve(seemps_ctx* ctx, const seemps_cgs_problem* problem,
                               const seemps_cgs_params* params, seemps_cgs_report* report);

#ifdef __cplusplus
}
#endif

#endif /* SEEMPS_GB300_H */
