/*
 * enmf.h -- C ABI of the GB300 exterior-NMF (eNMF) library, libenmf.so.
 *
 * The library computes the Frobenius-norm nonnegative factorisation
 *     minimise 1/2 ||X - U V^T||_F^2  subject to U >= 0, V >= 0      (Eq. 1)
 * with the exterior method of "An Exterior Method for Nonnegative Matrix
 * Factorization" (ICML 2026), Algorithm 3:
 *   1. enmf_svd_init  -- truncated SVD start U* = U_r S^(1/2), V* = V_r S^(1/2)
 *                        (Sec. 4; randomized range finder, Sec. 4.3 remark);
 *   2. enmf_rotate    -- orthogonal R toward the orthant by ADMM (Algorithm 1,
 *                        Eq. 7 prox, Procrustes R update, Sec. 4.1);
 *   3. enmf_iterate   -- ascent stage (Eq. 8/9 shifts + PBCD, Algorithm 2,
 *                        step sizes Eq. 10/11) until U, V >= 0, then HALS
 *                        descent (Sec. 4.3);
 *   4. enmf_residual  -- f(U, V) of Eq. 1 and ||X - UV^T||_F / ||X||_F;
 *   5. enmf_kkt       -- the KKT measures of App. G (Table 10).
 *
 * Conventions (App. I): X is m x n, U is m x r, V is n x r, X ~ U V^T.
 * All matrices are ROW-MAJOR.  X has leading dimension ldx >= n (elements);
 * U and V are dense with leading dimension r.
 *
 * Pointers: unless stated otherwise, matrix and vector arguments are DEVICE
 * pointers on the context's device, owned by the caller, and must stay valid
 * until the work enqueued on the context stream has finished.  X must be
 * aligned to 16 bytes.  The library never frees caller memory.
 *
 * Streams: every call enqueues its work on the stream given to enmf_create
 * (a cudaStream_t passed as void*; NULL = the legacy default stream).  Calls
 * that return host values (info structs, residuals, KKT reports) synchronise
 * that stream before returning; the others return as soon as the work is
 * enqueued.
 *
 * Errors: every call returns an enmf_status.  Arguments are checked before
 * any launch (ENMF_EINVAL, nothing enqueued).  Device-side failures (a
 * bounded wait that expired, a non-finite value) are reported through a
 * device status word read at the next synchronising call; after ENMF_ECUDA or
 * ENMF_ETIMEOUT the context is poisoned and later calls return that code.
 * No call throws, exits or falls back to host arithmetic.
 */
#ifndef ENMF_H
#define ENMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ENMF_OK = 0,
  ENMF_EINVAL = 1,      /* bad argument (shape, rank, dtype, null pointer)   */
  ENMF_EDOMAIN = 2,     /* X has a negative or non-finite entry               */
  ENMF_ENOMEM = 3,      /* device allocation failed                           */
  ENMF_ECUDA = 4,       /* a CUDA call failed; context poisoned               */
  ENMF_ETIMEOUT = 5,    /* a bounded device-side wait expired; poisoned       */
  ENMF_ENOTCONV = 6,    /* an iteration did not converge within its budget    */
  ENMF_EBUSY = 7,       /* context in use by another call                     */
  ENMF_ESTATE = 8       /* call out of order (e.g. rotate before svd_init)    */
} enmf_status;

/* Element types.  The "form" of a problem is (x_dtype, f_dtype, stream_dtype):
 *   plain FP64:  X F64, factors F64 (all arithmetic FP64);
 *   FP32:        X F32, factors F32 (FP32 arithmetic, FP64 scalar sums);
 *   BF16 / F16:  X BF16 or F16 (given, or staged from F32), factors F32; X
 *                products on the tensor cores with FP32 accumulation;
 *   FP8:         X F32 staged to E4M3 codes with per-tile scales, factors
 *                F32, tensor cores as for BF16. */
typedef enum { ENMF_F64 = 0, ENMF_F32 = 1, ENMF_BF16 = 2, ENMF_F16 = 3,
               ENMF_E4M3 = 4 /* stream type only: OCP FP8 E4M3 codes */,
               ENMF_CSR = 5  /* x_dtype only: X as compressed rows (enmf_csr) */ } enmf_dtype;

/* The sparse form (x_dtype = ENMF_CSR; the Reuters experiment of Sec. 5): X is
 * given by its stored entries.  Every call that takes X then takes a HOST
 * pointer to an enmf_csr whose three arrays are DEVICE memory of the caller:
 *   row_ptr  m + 1 entries, row_ptr[0] = 0, nondecreasing, row_ptr[m] = nnz;
 *   col      nnz column indices, strictly increasing within each row
 *            (row i's entries at row_ptr[i] .. row_ptr[i+1] - 1);
 *   val      nnz values, finite and >= 0, of the factors' type (FP64 with
 *            f_dtype = ENMF_F64, FP32 with ENMF_F32).
 * Entries not stored are zeros of X (this is not matrix completion).  The
 * first call with a new descriptor (new array pointers) checks it on the
 * device -- ENMF_EINVAL at that call for a malformed structure, ENMF_EDOMAIN
 * for a negative or non-finite value -- and builds the context's transpose
 * (compressed columns, each column's entries in row order); later calls with
 * the same pointers reuse it, so the arrays' contents must not change between
 * calls.  X V and X^T U then read the stored entries once each; the rest of
 * the method is unchanged.  Not available: the tensor-core forms, batches,
 * enmf_solve with host buffers, enmf_stage_x. */
typedef struct {
  const int64_t* row_ptr;
  const int32_t* col;
  const void* val;
} enmf_csr;

/* Largest supported rank (the SVD start works on r + oversample <= 80). */
#define ENMF_MAX_RANK 64

typedef struct {
  int64_t m;        /* rows of X, >= 1                                        */
  int64_t n;        /* columns of X, >= 1                                     */
  int64_t ldx;      /* row stride of X in elements, >= n                      */
  int32_t r;        /* rank, 1 <= r <= min(m, n, ENMF_MAX_RANK)               */
  int32_t x_dtype;  /* enmf_dtype of X                                        */
  int32_t f_dtype;  /* enmf_dtype of U and V: ENMF_F64 with X F64, else F32   */
  int32_t stream_dtype; /* type the iteration's X sweeps read:                */
                    /*   = x_dtype (or 0 with F64 X): the SIMT sweeps;        */
                    /*   ENMF_BF16 / ENMF_F16 with F32 X: the precision form  */
                    /*   -- the tensor-core sweeps read X_hi = t(X) and apply */
                    /*   X_lo = t(X - X_hi) every correct_every steps, t the  */
                    /*   rounding to that type (FP16: X <= 65504, else        */
                    /*   ENMF_EDOMAIN at enmf_stage_x's next sync);           */
                    /*   ENMF_BF16 / ENMF_F16 with X of that type: tensor-    */
                    /*   core sweeps on X as given (no correction).  F32      */
                    /*   factors required; with FP16 the factor entries must  */
                    /*   stay within the FP16 range.                          */
                    /*   ENMF_E4M3 with F32 X: the FP8 form -- X_hi is e4m3   */
                    /*   codes with a power-of-two scale per 128 x 128 tile   */
                    /*   and X_lo = bf16(X - X_hi) (see enmf_stage_x); X must */
                    /*   stay <= 448 * 2^100; m <= 65535 * 128.               */
  int64_t nnz;      /* ENMF_CSR: stored entries (0 <= nnz <= m n; m, n and    */
                    /*   nnz below 2^31); ldx is then ignored.  Else unused.  */
} enmf_problem;

typedef struct enmf_ctx enmf_ctx;

/* Bytes of device workspace a context for *p allocates (for admission by
 * memory footprint; X, U and V are the caller's and not included). */
enmf_status enmf_workspace_size(const enmf_problem* p, size_t* bytes);

/* Create a context on the current device.  Allocates the workspace (owned by
 * the context, freed by enmf_destroy).  `stream` is a cudaStream_t or NULL. */
enmf_status enmf_create(const enmf_problem* p, void* stream, enmf_ctx** out);
void enmf_destroy(enmf_ctx* ctx);
const char* enmf_status_string(enmf_status s);

/* ---- 1. SVD start (Sec. 4) ---------------------------------------------
 * Randomized subspace iteration with oversampling p: Q spans X*Omega, then
 * alternately X^T Q and X Q2 are orthonormalised (two passes of T = D L^-T from
 * the Cholesky factor L of the diagonally scaled Gram D G D; a Gram eigen map
 * with numerical-rank truncation when a pivot is near zero) and the top-r Ritz
 * triplets of the Rayleigh-Ritz matrix are taken by one-sided Jacobi SVD in
 * FP64.  Iterates
 * until ||X V_r - U_r S_r||_F <= tol * sigma_1, at most max_iters times.
 * Output: U (m x r) = U_r S^(1/2), V (n x r) = V_r S^(1/2), with column j of
 * both negated when sum_i U_ij + sum_i V_ij < 0; sigma (device, r doubles)
 * = the top r singular values, descending.  Omega's entries are
 * uniform(-1, 1) from a counter-based hash of (seed, i, j).
 * Returns ENMF_ENOTCONV (outputs still written) if tol is not met. */
typedef struct {
  int32_t oversample;   /* p, default 10                                   */
  int32_t max_iters;    /* default 40                                      */
  double tol;           /* default 1e-12 (FP32 factors: 1e-5)              */
  uint64_t seed;        /* default 0x5eed                                  */
  int32_t fp32_finish;  /* FP32 factors: 1 = the start from the FP32       */
                        /*   Jacobi SVD of the last Rayleigh-Ritz matrix   */
                        /*   (the one the stopping test used); 0 (default) */
                        /*   = that SVD finished by FP64 sweeps            */
} enmf_svd_opts;
typedef struct {
  int32_t iters;        /* power iterations taken                          */
  int32_t rank;         /* numerical rank kept (<= r + oversample)         */
  double residual;      /* ||X V_r - U_r S_r||_F / sigma_1 at exit          */
} enmf_svd_info;
enmf_status enmf_svd_init(enmf_ctx* ctx, const void* X, void* U, void* V, double* sigma,
                          const enmf_svd_opts* opts /* NULL = defaults */,
                          enmf_svd_info* info /* NULL ok */);

/* The SVD start for `count` contexts at once (no counterpart in the paper; a
 * serving aid): each problem exactly as enmf_svd_init(ctxs[i], X[i], U[i],
 * V[i], sigma ? sigma[i] : NULL, opts, &infos[i]) would leave it, bit for
 * bit.  The problems' power iterations run in lockstep, each problem's kernels
 * in its own order; the single-CTA steps of all problems (the range finder's
 * Gram eigen maps, the stopping test's Rayleigh-Ritz SVDs and the
 * FP32-then-FP64 SVDs that finish the FP32-factor starts) run in one launch
 * each, one CTA per problem, and one synchronisation per power iteration
 * serves every stopping test.  All contexts must share
 * one stream and device and appear once (else ENMF_EINVAL, before any
 * launch); forms may differ.  status (may be NULL) receives each problem's
 * status (ENMF_OK or ENMF_ENOTCONV as enmf_svd_init returns them); the call
 * returns the first status other than those, else ENMF_OK. */
enmf_status enmf_svd_init_group(enmf_ctx* const* ctxs, const void* const* X, void* const* U,
                                void* const* V, double* const* sigma, int32_t count,
                                const enmf_svd_opts* opts, enmf_svd_info* infos,
                                enmf_status* status);

/* ---- 2. Rotation toward the orthant (Algorithm 1) -----------------------
 * W = [U; V].  Each ADMM step: b = W R - Y / rho; Z = prox(b) (Eq. 7);
 * M = W^T (Z + Y / rho); R = polar(M) = C D^T from M = C S D^T (Procrustes;
 * FP64 factors: warm-started one-sided Jacobi SVD in FP64; FP32 factors:
 * Newton-Schulz in FP32 with a last step on X^T X formed in FP64, every step
 * of the loop in one persistent launch); Y += rho (Z - W R).  R0 = I, Y0 = 0.
 * rho = rho_scale / RMS(W) unless rho > 0 is given.  Stops when
 * ||R_k+1 - R_k||_F <= tol * sqrt(r) or after max_iter steps.  On exit U and V
 * are overwritten in place by U R and V R; R (device, r x r row-major FP64)
 * receives R if non-NULL.  Resets the iteration state (a new ascent stage). */
typedef struct {
  double rho;           /* <= 0: use rho_scale / RMS(W)                    */
  double rho_scale;     /* default 3                                       */
  int32_t max_iter;     /* default 200                                     */
  double tol;           /* default 1e-12                                   */
  int32_t f64;          /* FP32 factors: 1 = run the ADMM in FP64 (rows    */
                        /*   and r x r update) on FP64 copies of U*, V*,   */
                        /*   the rotated factors rounded to FP32 once; 0   */
                        /*   (default) = the FP32 persistent kernel        */
} enmf_admm_opts;
typedef struct {
  int32_t steps;
  int32_t converged;
  double rho;
  double dR;            /* ||R_k+1 - R_k||_F of the last step               */
  double neg_mass_in;   /* sum h(W) before                                  */
  double neg_mass_out;  /* sum h(W R) after                                 */
} enmf_rotate_info;
enmf_status enmf_rotate(enmf_ctx* ctx, void* U, void* V, double* R,
                        const enmf_admm_opts* opts, enmf_rotate_info* info);

/* The rotation of Algorithm 1 for `count` problems at once (no counterpart in
 * the paper; a serving aid): ctxs[i] with its factors U[i], V[i] (device),
 * each exactly as enmf_rotate(ctxs[i], U[i], V[i], NULL, opts, &infos[i])
 * would leave them, bit for bit, but the FP32 ADMM steps of many problems
 * run in one cooperative grid: problem i gets the blocks its own launch
 * would have, its polar factor is formed on its own first block, so the
 * per-step polar factors of the problems are formed side by side.  Problems
 * are packed into as few grids as the device holds.  Every context must have
 * FP32 factors, the same rank pad (16, 32, 48 or 64) and the same stream;
 * opts->f64 must be 0; no context may appear twice (else ENMF_EINVAL, before
 * any launch).  infos (may be NULL) receives count records.  Synchronises
 * twice per call (the rho inputs, then the results).  Returns the first
 * non-OK status of the problems in order; ENMF_ENOTCONV (a polar iteration
 * that did not settle) leaves results and infos as enmf_rotate does, a
 * device-side failure poisons the contexts whose problems it concerns. */
enmf_status enmf_rotate_group(enmf_ctx* const* ctxs, void* const* U, void* const* V,
                              int32_t count, const enmf_admm_opts* opts,
                              enmf_rotate_info* infos);

/* ---- 2b. Generalized rotation (Eq. 5, Algorithm 4, App. A.2) -----------
 * Orthogonal R1, R2 and diagonal Lambda > 0 that bring U* R1 Lambda R2 and
 * V* R1 Lambda^-1 R2 toward the orthant (the product U V^T is unchanged).
 * ADMM with the splitting W1 = W_svd R1, W2 = [W11 Lambda; W12 Lambda^-1],
 * W3 = W2 R2 and scaled duals M, N, P; one step, in the order of Algorithm 4:
 * W3 = prox(W2 R2 - P) (the Eq. 7 form), W1 and W2 from their closed forms,
 * R1 = polar(W_svd^T (W1 + M)), R2 = polar(W2^T (W3 + P)) (FP64 Jacobi),
 * lambda_i = the positive root of a l^4 - b l^3 + c l - d = 0 (App. A.2)
 * with the least objective, then the dual updates.  Start: R1 = R2 = I,
 * Lambda = I, W1 = W2 = W3 = W_svd, zero duals; rho = gamma = t =
 * rho_scale / RMS(W) unless opts->rho > 0.  Stops when |R1 - R1'| + |R2 -
 * R2'| + |lambda - lambda'| <= tol sqrt(r) (Frobenius norms) or after
 * max_iter steps (the step count is exact: a device flag skips the steps
 * enqueued after the rule holds).  U and V are overwritten by the rotated
 * factors; R1, R2 (r x r row-major) and lam (r) are device FP64 outputs;
 * info->dR is the last step's change.  The workspace (6 (m + n) r elements
 * plus small buffers) comes from the stream-ordered allocator for the call.
 * Resets the iteration state.  Synchronises. */
enmf_status enmf_rotate_general(enmf_ctx* ctx, void* U, void* V, double* R1, double* lam,
                                double* R2, const enmf_admm_opts* opts, enmf_rotate_info* info);

/* ---- 3. Exterior iteration (Algorithm 3 lines 5-12) ---------------------
 * Runs n_iter alternations from the context's iteration state.  One
 * alternation = U-half then V-half.  While U or V has a negative entry it is
 * an ascent step: negative entries += s (Eq. 8/9; s = max(-F) / (n_shift -
 * 1/2), fixed at the first ascent step), mask M+ = [F >= 0], then PBCD
 * (Algorithm 2) with d_i = ||g_i||^2 / (g_i G g_i^T) (Eq. 10/11), stopping at
 * ||M+ o grad|| < eps ||grad_init|| or pbcd_max_iter sweeps.  Afterwards it is
 * a HALS sweep of U's columns then V's columns.  Each alternation reads X
 * once for X V and once for X^T U (in the HALS stage of the tensor-core
 * forms optionally once for both, see enmf_set_fused).  trace (device, FP64, n_iter entries, may
 * be NULL) receives f(U, V) of Eq. 1 after every V-half, from the expansion
 * 1/2 ||X||^2 - <X^T U, V> + 1/2 <U^T U, V^T V> summed in FP64. */
typedef struct {
  int32_t n_iter;         /* alternations to run, >= 0                     */
  int32_t pbcd_max_iter;  /* default 5                                     */
  double eps;             /* default 1e-4                                  */
  int32_t n_shift;        /* default 3                                     */
  double* trace;          /* device FP64 [n_iter] or NULL                  */
  int32_t reset;          /* 1: start a new ascent stage from (U, V)       */
  int32_t sync_info;      /* 1: synchronise and fill *info                 */
  int32_t correct_every;  /* precision form: refresh X_lo V and X_lo^T U   */
                          /* every this many alternations (default 10)     */
} enmf_iter_opts;
typedef struct {
  int32_t iters;          /* alternations done in total (this state)       */
  int32_t asc_iters;      /* of which ascent steps                         */
  int32_t hals_iters;     /* of which HALS steps                           */
  int32_t stage;          /* 0 ascent, 1 HALS                              */
  double s_u, s_v;        /* shift steps of Eq. 8 / 9                      */
} enmf_iter_info;
enmf_status enmf_iterate(enmf_ctx* ctx, const void* X, void* U, void* V,
                         const enmf_iter_opts* opts, enmf_iter_info* info);

/* PBCD sweep counts of the ascent steps run so far: out[2k] (U-half) and
 * out[2k+1] (V-half) for ascent step k; *count = number of ascent steps.
 * Host buffer of `cap` ints.  Synchronises. */
enmf_status enmf_pbcd_counts(enmf_ctx* ctx, int32_t* out, int32_t cap, int32_t* count);

/* ---- 4. Residual (Eq. 1) -------------------------------------------------
 * out[0] = f = 1/2 ||X - U V^T||_F^2, out[1] = ||X - U V^T||_F / ||X||_F,
 * out[2] = ||X||_F^2 (host doubles).  direct = 1: one pass over X forming each
 * entry of X - U V^T (FP64 sums); direct = 0: the Gram expansion.  Syncs. */
enmf_status enmf_residual(enmf_ctx* ctx, const void* X, const void* U, const void* V,
                          double* out3, int32_t direct);

/* ---- 5. KKT measures (App. G, Eq. kkt-nmf, Table 10) ---------------------
 * grad_U = U (V^T V) - X V, grad_V = V (U^T U) - X^T U; W stacks U over V.
 * delta = max(grad_W o W), sigma = sum(grad_W o W), min W, min grad_W, the
 * projected-gradient norm (grad where W > 0, min(0, grad) where W = 0) and
 * that norm over ||XV|| + ||U V^T V|| + ||X^T U|| + ||V U^T U||.  Syncs. */
typedef struct {
  double min_w, min_grad, delta, sigma, pg_norm, pg_rel;
} enmf_kkt_report;
enmf_status enmf_kkt(enmf_ctx* ctx, const void* X, const void* U, const void* V,
                     enmf_kkt_report* out);

/* ---- Tensor-core staging (precision form) --------------------------------
 * With stream_dtype = ENMF_BF16, stage X once before svd_init / iterate /
 * sweep: F32 X is split into context-owned X_hi = bf16(X) and
 * X_lo = bf16(X - X_hi) (row stride rounded up to 8 elements) and TMA
 * descriptors are built; BF16 X is used in place (it must be 16-byte aligned
 * with ldx a multiple of 8).  Later calls must pass the same X pointer
 * (ENMF_ESTATE otherwise).  ENMF_EDOMAIN if X has a negative or non-finite
 * entry.  Enqueued on the context stream. */
enmf_status enmf_stage_x(enmf_ctx* ctx, const void* X);
/* With stream_dtype = ENMF_E4M3 (the FP8 form, with per-tile scaling; no
 * counterpart in the paper), staging splits F32 X per 128 x 128 tile
 * (I, J) -- the last tiles of a ragged X are partial:
 *   k_IJ = the least integer with max(tile) <= 448 * 2^k, at least -100;
 *   q = e4m3(x * 2^-k) rounded to nearest even, with codes below 8 (values
 *       under 2^-6, the E4M3 subnormals) replaced by 0;
 *   X_hi = q * 2^k (exact in BF16), X_lo = bf16(x - X_hi), round to nearest
 *       even.
 * The sweeps stream the one-byte codes; X_lo is applied like the 16-bit
 * forms' X_lo.  ENMF_EDOMAIN (at the next sync) for a negative or non-finite
 * entry, or one beyond 448 * 2^100.
 *
 * enmf_stage_copy copies the staged decomposition of the tensor-core forms
 * to caller buffers (device or host, told apart by the CUDA runtime; any may
 * be NULL) and synchronises the context stream: hi = X_hi as m x n dense
 * elements (BF16 / FP16 bits, or e4m3 codes), lo = X_lo as m x n dense
 * 16-bit elements, tile_exp = the ceil(m/128) x ceil(n/128) exponents k
 * (FP8 form only).  ENMF_ESTATE before staging; ENMF_EINVAL for a buffer the
 * form does not have (lo with 16-bit X given as is, tile_exp outside the FP8
 * form).  For inspection and tests; no counterpart in the paper. */
enmf_status enmf_stage_copy(enmf_ctx* ctx, void* hi, void* lo, int32_t* tile_exp);

/* ---- The core NMF kernel (App. I): X V and X^T U --------------------------
 * XV (m x r) = X V and XtU (n x r) = X^T U in the context's form, FP32 or
 * FP64 like the factors, device pointers, row-major with leading dimension r.
 * Either output may be NULL.  Precision form: exact = 1 adds the X_lo terms
 * (two passes), exact = 0 uses X_hi only.  Enqueued, no sync. */
enmf_status enmf_sweep(enmf_ctx* ctx, const void* X, const void* U, const void* V, void* XV,
                       void* XtU, int32_t exact);

/* ---- One call, host or device buffers -------------------------------------
 * The whole of Algorithm 3: svd_init, rotate, iterate(n_iter), residual.  X,
 * U and V may be host or device pointers (told apart by the CUDA runtime);
 * host data is copied through context-owned device buffers inside the call.
 * out3 as for enmf_residual (host).  NULL opts = defaults.  Syncs. */
enmf_status enmf_solve(enmf_ctx* ctx, const void* X, void* U, void* V, int32_t n_iter,
                       const enmf_svd_opts* svd, const enmf_admm_opts* admm,
                       const enmf_iter_opts* iter, double* out3);

/* ---- Batching (no counterpart in the paper) --------------------------------
 * A batch iterates many independent problems together.  Each phase of every
 * alternation is one grouped launch over all members: X V sweep, U-half,
 * X^T U sweep, V-half (plus the X_lo passes every correct_every
 * alternations).  The sweeps run stream-K over the members' concatenated
 * tensor-core work.  The half steps run each member on its own group of blocks
 * of one cooperative grid.  A step of n_alt alternations is captured as a CUDA
 * graph and replayed while the membership is unchanged.
 *
 * Members are contexts of the tensor-core form (stream_dtype ENMF_BF16, FP32
 * factors) with X staged, whose U and V (device, caller-owned) are the
 * starting point -- normally the output of enmf_svd_init and enmf_rotate.
 * A context of the FP8 form (stream_dtype ENMF_E4M3) is rejected with
 * ENMF_EINVAL: it iterates alone.
 * All members of a batch share the padded rank (r rounded up to 16, 32, 48
 * or 64); a member of another padded rank is rejected with ENMF_EINVAL.
 * The iteration options (pbcd_max_iter, eps, n_shift, correct_every; the
 * trace, reset and sync_info fields are ignored) are fixed at creation.
 *
 * enmf_batch_add starts the member's iteration (state reset, as enmf_iterate
 * with reset = 1) on the member's stream; the batch stream waits for it.
 * ENMF_EBUSY: no free slot, or the grouped half step would exceed the
 * co-resident capacity.  enmf_batch_remove makes the member's stream wait
 * for the batch's work; U and V then hold the member's iterate.  Neither
 * call synchronises.  A removed context may be destroyed or added again.
 * enmf_batch_step enqueues n_alt alternations of every member on the batch
 * stream; n_alt must be a multiple of correct_every (ENMF_EINVAL otherwise),
 * so every member joins at the start of a correction period and refreshes
 * its X_lo terms at the same alternations as it would alone.  enmf_batch_member synchronises the batch stream and reports a
 * member's alternation count, stage and objective f (Eq. 1) after its last
 * alternation.  enmf_batch_tune times the grouped sweeps of the current
 * membership at several stream-K grid sizes (a quarter, half, three quarters
 * and all of the SMs) and depths of their shared-memory ring of X stages (2,
 * 3, or as deep as fits) and keeps the fastest pair (*grid, and the time of
 * one X V + X^T U pair in ms); it synchronises.  The serving loop re-tunes
 * when a batch's membership has changed by half since the last tuning.  A context
 * may be in one batch at a time, and must not be used by other calls while
 * it is a member. */
typedef struct enmf_batch enmf_batch;
enmf_status enmf_batch_create(const enmf_iter_opts* opts /* NULL = defaults */,
                              int32_t max_members, void* stream, enmf_batch** out);
void enmf_batch_destroy(enmf_batch* b);
enmf_status enmf_batch_add(enmf_batch* b, enmf_ctx* ctx, const void* X, void* U, void* V,
                           int32_t* slot);
enmf_status enmf_batch_remove(enmf_batch* b, int32_t slot);
int32_t enmf_batch_size(const enmf_batch* b);
enmf_status enmf_batch_step(enmf_batch* b, int32_t n_alt);
enmf_status enmf_batch_member(enmf_batch* b, int32_t slot, enmf_iter_info* info, double* f);
enmf_status enmf_batch_tune(enmf_batch* b, int32_t* grid, float* ms);
/* Every member's state at once (one synchronisation and one copy instead of
 * one per member): *count = members; for i < *count, slots[i], infos[i] and
 * f[i] as enmf_batch_member gives them.  Host arrays of cap entries;
 * ENMF_EINVAL when cap < *count (nothing written but *count). */
enmf_status enmf_batch_states(enmf_batch* b, int32_t* slots, enmf_iter_info* infos, double* f,
                              int32_t cap, int32_t* count);

/* ---- Checkpoint of the iteration state (no counterpart in the paper) -----
 * Algorithm 3's loop carries state between alternations, beside U and V:
 *   - the stage (ascent, lines 5-11, or HALS, line 12);
 *   - the fixed shift steps of Eq. 8 / 9 and the negative maxima they came from;
 *   - the alternation counters and the last objective.
 * enmf_state_export writes that state into a host buffer of ENMF_STATE_BYTES
 * bytes. The buffer is a fixed little-endian layout, versioned, carrying the
 * problem's sizes and types. enmf_state_import loads such a buffer into a
 * context of the same problem; enmf_iterate with reset = 0 then continues the
 * iteration from the caller's U and V (which the caller saves and restores
 * itself) as the exporting context would have.
 * Both synchronise the context stream.
 * enmf_state_export: *bytes >= ENMF_STATE_BYTES on entry (set to the size
 * written on return); ENMF_ESTATE when no iteration has run since the last
 * svd_init / rotate (nothing to export).
 * enmf_state_import: ENMF_EINVAL for a short buffer, an unknown layout or a
 * different problem (m, n, r, types). */
#define ENMF_STATE_BYTES 128
enmf_status enmf_state_export(enmf_ctx* ctx, void* buf, size_t* bytes);
enmf_status enmf_state_import(enmf_ctx* ctx, const void* buf, size_t bytes);

/* ---- Measurement (no counterpart in the paper) ---------------------------
 * enmf_profile: every > 0 records CUDA events around the X V and X^T U sweep
 * kernels (the main pass over X alone: not the factor split or the X_lo
 * correction pass) of every `every`-th alternation in enmf_iterate (on the
 * context stream, up to 128 alternations per call); 0 turns it off.  enmf_profile_read returns
 * the summed sweep time (ms) and the number of timed sweeps, optionally
 * resetting them; it synchronises the stream.
 * enmf_probe_fma_peak: measured FMA throughput (flop/s) of the current device
 * for ENMF_F64 or ENMF_F32 (a throughput kernel timed with CUDA events).
 * enmf_launch_count: kernel launches issued by the library since load. */
enmf_status enmf_profile(enmf_ctx* ctx, int32_t every);
enmf_status enmf_profile_read(enmf_ctx* ctx, double* sweep_ms, int64_t* sweeps, int32_t reset);
enmf_status enmf_probe_fma_peak(int32_t dtype, double* flops_per_s);
long long enmf_launch_count(void);

/* ---- Equivalence of two factorisations (Sec. 5, App. F and App. H) -------
 * Both take factor matrices of the context's problem and form (m x r and
 * n x r, row-major, device, f_dtype); the context gives the stream and the
 * scratch.  Both synchronise.
 *
 * enmf_equiv_transform (App. F): R1, Lambda, R2 with
 *     U_alg ~ U_e R1 Lambda R2^T,   V_alg ~ V_e R1 Lambda^-1 R2^T,
 * from the least-squares map Z = (U_e^T U_e)^-1 U_e^T U_alg (the paper's
 * Q Gamma^-1 P^T U_alg for the SVD U_e = P Gamma Q^T) and its SVD
 * Z = R1 Lambda R2^T.  R1, R2 (r x r row-major) and lam (the diagonal of
 * Lambda, descending) are device FP64 buffers; delta2 (host, 2 doubles)
 * receives delta_u = ||U_alg - U_e Z||_F and delta_v = ||V_alg - V_e
 * R1 Lambda^-1 R2^T||_F (both 0 when the factorisations are equivalent).
 * ENMF_ENOTCONV when U_e^T U_e is not positive definite (U_e rank deficient).
 *
 * enmf_perm_check (App. H): the columns of U_B that are scaled permutations
 * of columns of U_A.  Pairs (i, j) are taken one to one in decreasing
 * cos(U_A^(i), U_B^(j)) (ties by lower i, then j) while the cosine is
 * >= 1 - eps (the paper uses eps = 0.05); then, on the candidates, the
 * columns of the self-similarity matrices of U_A's and U_B's candidates and
 * of their cross-similarity matrix are sorted in descending order and
 * rounded to one decimal (floor(10 x + 1/2)), and a candidate stays when its
 * column agrees in all three at more than keep_frac of the positions (the
 * paper uses 0.9).  b_of_a (host, r ints) receives for each column i of U_A
 * the matched column of U_B, or -1; *kept the number of pairs. */
enmf_status enmf_equiv_transform(enmf_ctx* ctx, const void* Ue, const void* Ve, const void* Ua,
                                 const void* Va, double* R1, double* lam, double* R2,
                                 double* delta2);
enmf_status enmf_perm_check(enmf_ctx* ctx, const void* UA, const void* UB, double eps,
                            double keep_frac, int32_t* b_of_a, int32_t* kept);

/* ---- Matrix completion (App. C, Algorithm eNMC) ---------------------------
 * For a context of the sparse form (x_dtype = ENMF_CSR, X an enmf_csr): here
 * the stored entries are the KNOWN entries of X (the mask M_E) and the others
 * are unknown, not zeros.  The objective is
 *     f^(U, V) = 1/2 ||M_E o (X - U V^T)||_F^2.
 * Algorithm eNMC is enmf_nmc_start, enmf_rotate (Algorithm 1 unchanged), then
 * enmf_nmc_iterate.  Other forms: ENMF_ESTATE.
 *
 * enmf_nmc_start: the unconstrained start (App. C computes a local minimum of
 * f^ with softImpute-ALS): from the balanced truncated SVD of the zero-filled
 * X (enmf_svd_init), sweeps of exact row least squares with softImpute's
 * ridge, every row of U then every row of V,
 *     u_i = (G_i + lam c_i I)^-1 a_i,  G_i = sum over known (i, j) of v_j v_j^T,
 *     a_i = sum over known (i, j) of x_ij v_j,  c_i = trace(G_i) / r (1 if 0),
 * G_i and a_i formed and solved (Cholesky) in FP64 in every form, until f^
 * changes by <= tol (relative) over a sweep or after max_sweeps sweeps.  The
 * ridge makes the rows with fewer known entries than r well posed (their G_i
 * is singular).  Overwrites U, V.  info (may be NULL): sweeps run and the
 * final f^.  ENMF_ENOTCONV when a row's matrix was not positive definite in
 * FP64 (lam = 0 and a row with fewer than r known entries).
 *
 * enmf_nmc_iterate: opts->n_iter rounds of Algorithm eNMC: shift U's negative
 * entries (Eq. 8, step fixed when the state is reset, as in enmf_iterate),
 * mask M+ = [U >= 0], PBCD on U's rows with M_E (Algorithm 2):
 *     g_i = M+ o (u_i G_i - a_i),  d_i = ||g_i||^2 / (g_i G_i g_i^T)
 * -- the exact minimiser of f^ along -g_i, Eq. 10 when every entry is known --
 * u_i <- max(0, u_i - d_i g_i) on the mask, stopping when ||g|| < eps
 * ||g_init|| (all rows) or after pbcd_max_iter sweeps; then the same for V
 * with M_E^T.  G_i and a_i are formed once per half from the stored entries.
 * opts->trace (device FP64, n_iter, may be NULL) receives f^ after every
 * round; reset = 1 restarts (new shift steps from the current U, V).  The
 * work buffers (max(m, n) r_pad^2 + max(m, n) r_pad elements, r_pad = r
 * rounded up to 16, 32, 48 or 64) come from the stream-ordered allocator.
 * info: iters = asc_iters = rounds since the reset, s_u, s_v.
 *
 * enmf_nmc_objective: out2[0] = f^, out2[1] = ||M_E o (X - U V^T)||_F /
 * ||M_E o X||_F (host, 2 doubles).  Synchronises. */
typedef struct {
  int32_t max_sweeps;   /* default 50                                      */
  double lam;           /* default 1e-3                                    */
  double tol;           /* default 1e-10                                   */
  int32_t svd_max_iters;/* the SVD start's max_iters; 0 = its default      */
} enmf_nmc_start_opts;
typedef struct {
  int32_t sweeps;
  double f;
} enmf_nmc_start_info;
enmf_status enmf_nmc_start(enmf_ctx* ctx, const void* X, void* U, void* V,
                           const enmf_nmc_start_opts* opts, enmf_nmc_start_info* info);
enmf_status enmf_nmc_iterate(enmf_ctx* ctx, const void* X, void* U, void* V,
                             const enmf_iter_opts* opts, enmf_iter_info* info);
enmf_status enmf_nmc_objective(enmf_ctx* ctx, const void* X, const void* U, const void* V,
                               double* out2);

/* ---- The fused single-pass alternation (no counterpart in the paper) -----
 * In the HALS stage of the BF16 / FP16 tensor-core forms (rank padded to 32
 * or 64, and X narrow enough that a cluster of CTAs holds V's column slices
 * in shared memory: n up to about 12,000 at rank pad 32), enmf_iterate runs
 * each alternation as one pass over X: per 128-row panel, X V, the HALS
 * update of the panel's rows of U (Sec. 4.3) and X_panel^T U_new for the
 * V-half, so X is read once per alternation instead of twice.  From a fresh
 * ascent stage the first n_shift alternations (the ascent stage, which ends
 * within them) use the two-pass sweeps, and the call then synchronises once
 * to read the stage.  The fused pass is OFF by default: on a GB300 its
 * exchange across the cluster for every 128-row panel is latency-bound, and
 * at the measured shapes the two-pass sweeps are faster.  enmf_set_fused(ctx,
 * 1) turns it on, 0 off; *available (may be NULL) tells whether the context
 * can run it at all. */
enmf_status enmf_set_fused(enmf_ctx* ctx, int32_t on, int32_t* available);

/* ---- Overlap of consecutive kernels (no counterpart in the paper) ---------
 * In the captured alternation loop of the tensor-core forms, a kernel may be
 * launched as a programmatic dependent of the one before it: it starts while
 * that kernel still runs, and waits for its completion before touching
 * anything it shares with it.  flags bit 0: each X sweep after a half step
 * (its CTAs request their first X tiles early; X is not written inside the
 * loop); bit 1: each half step after a sweep (its launch overlaps the sweep's
 * last CTAs).  Results are bit-identical either way.  Default 1: on a GB300
 * (dense 8192 x 6144, r = 32, 500 alternations) bit 0 took 40.3 ms against
 * 40.7 ms without, bit 1 41.9 ms and both 45.3 ms (a half step's blocks that
 * start early run on SMs whose shared memory is configured for the sweep,
 * with less L1 cache).  flags < 0
 * leaves the setting unchanged; flags > 3 is ENMF_EINVAL.  *in_effect (may be
 * NULL) receives the flags in effect: a capture that the driver refuses with
 * the attribute is redone without it and the flags drop to 0. */
enmf_status enmf_set_overlap(enmf_ctx* ctx, int32_t flags, int32_t* in_effect);
/* The fused pass's launch shape, for reports: shape[0] = 1 if available,
 * shape[1] = CTAs per cluster, [2] = clusters, [3] = columns of X per CTA,
 * [4] = X stages in shared memory, [5] = dynamic shared memory per CTA (KB). */
enmf_status enmf_fused_shape(enmf_ctx* ctx, int32_t* shape);
/* Diagnostics: with the environment variable ENMF_FUSED_STAMPS set when the
 * context is created, the fused pass records %globaltimer stamps (ns) of its
 * phases, per CTA and panel, overwritten by every launch.  *count receives the
 * number of 64-bit stamps; they are copied to the host buffer out when
 * cap >= *count (then the call synchronises).  Layout: stamp e (0..7) of local
 * panel p of CTA c at (c (P + 1) + p) 8 + e, P = 32 (later panels are not
 * recorded); panel slot P holds the CTA's start (e = 0) and end (e = 1).  Events: 0 X V
 * accumulator ready, 1 every CTA staged its partial, 2 rows summed, 3 HALS
 * done, 4 panel buffer free, 5 rows pushed, 6 (MMA thread) panel's U ready,
 * 7 X^T U issued.  *count = 0 when not recording. */
enmf_status enmf_fused_stamps(enmf_ctx* ctx, long long* out, int64_t cap, int64_t* count);

/* ---- Bounded device waits (no counterpart in the paper) ------------------
 * Every device-side wait of the library is bounded; an expired wait records
 * a timeout in the context's status word, the kernel goes on without the
 * awaited data (results are then meaningless, never out of bounds), and the
 * next synchronising call returns ENMF_ETIMEOUT and poisons the context.
 * enmf_set_wait_limit sets the spin limit, in SM clock cycles, of the grid
 * barriers of the context's cooperative kernels (half steps, PBCD stop test,
 * ADMM loop): 0 restores the default (about 2 s); at most 4e9.  A small
 * limit makes barriers expire on purpose: for tests of the failure path and
 * for callers that prefer an early error to a long stall.  Synchronises.
 * enmf_probe_wait launches one thread that waits, bounded by `cycles`, for
 * an event that never occurs -- kind 0: a global flag that nothing sets (the
 * barriers' spin); kind 1: a shared-memory mbarrier phase that nothing
 * completes (the tensor-core sweeps' pipeline waits) -- and sets *status to
 * ENMF_ETIMEOUT when the wait gave up as it must (ENMF_OK otherwise).  It
 * uses no context; the CUDA context stays usable.  Synchronises the device. */
enmf_status enmf_set_wait_limit(enmf_ctx* ctx, int64_t cycles);
enmf_status enmf_probe_wait(int32_t kind, int64_t cycles, int32_t* status);

/* ---- Allocation-free residual (no counterpart in the paper) --------------
 * The paper has no such call.  enmf_residual_noalloc computes the three
 * numbers of enmf_residual with direct = 1:
 *   out3[0] = f = 1/2 ||X - U V^T||_F^2,
 *   out3[1] = ||X - U V^T||_F / ||X||_F   (0 when ||X|| = 0),
 *   out3[2] = ||X||_F^2,
 * without a context and without allocating any memory.
 *
 * Who needs it.  Two kinds of callers cannot allocate, so they cannot use
 * enmf_create.  First, a caller whose device memory is already committed: a
 * large X and a running solve's workspace can fill the device, and then any
 * allocation may fail in the middle of a run.  Second, a caller that must not
 * stall other streams: cudaFree synchronises the whole device, and a caching
 * allocator may free memory at any time.  An example is a monitor that checks
 * factors written by a solve on another stream while that solve runs.
 *
 * Arguments.  X is m x n, row-major, with row stride ldx >= n elements, of
 * type x_dtype.  U (m x r) and V (n x r) are dense, row-major, of type f_dtype.
 * The forms are those of enmf_problem: ENMF_F64 factors need ENMF_F64 X;
 * ENMF_F32 factors take X of type ENMF_F32, ENMF_BF16 or ENMF_F16.  X, U, V and
 * out3 are DEVICE pointers on the current device, owned by the caller.  out3
 * receives 3 doubles.  stream is a cudaStream_t passed as void* (NULL = the
 * legacy default stream).  The call only enqueues work and does not
 * synchronise: out3 holds the result once the stream reaches the work.  The
 * sign of X is not checked.  m = 0 or n = 0 gives {0, 0, 0}.  The arithmetic
 * matches enmf_residual with direct = 1 except for the order of the FP64 sums.
 *
 * Limits.  m <= ENMF_RESIDUAL_NOALLOC_MAX_ROWS (4096 panels of 64 rows each)
 * and 1 <= r <= ENMF_MAX_RANK.  A larger m, or any other bad argument, returns
 * ENMF_EINVAL before anything is enqueued.  The current device index must be
 * below 64 (ENMF_EINVAL otherwise).
 *
 * Scratch.  The call sums through one fixed array in the library's static
 * device memory: 65,792 bytes per device (two FP64 sums per panel and one
 * arrival counter).  The counter must start at zero, so each call clears it
 * on `stream` before its kernel.  Nothing else needs clearing.
 *
 * Set-up.  The first call on each device, made with that device current, does
 * one-time set-up: it looks up the scratch array's address and loads the
 * kernels.  Make that first call before any stream capture.  Later calls only
 * enqueue a memset and one kernel.
 *
 * Concurrency.  All calls on one device share the same scratch.  Calls that
 * overlap on the device race on it and give wrong results.  Overlap happens
 * with calls on different streams that no event orders, or with calls from
 * several host threads.  Put such calls on one stream, or order them with
 * events.
 *
 * Errors: ENMF_EINVAL as above; ENMF_ECUDA if the set-up, the memset or the
 * launch fails.  A fault while the kernel runs shows up at the caller's next
 * synchronisation. */
#define ENMF_RESIDUAL_NOALLOC_MAX_ROWS 262144
enmf_status enmf_residual_noalloc(const void* X, int32_t x_dtype, int64_t m, int64_t n,
                                  int64_t ldx, const void* U, const void* V, int32_t r,
                                  int32_t f_dtype, double* out3, void* stream);

/* Library version string. */
const char* enmf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ENMF_H */
