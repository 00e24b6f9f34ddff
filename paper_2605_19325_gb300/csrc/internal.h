// Internal declarations shared by the library's translation units: the
// device-resident iteration state, the context, and the host-side launchers.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/enmf.h"
#include "common.cuh"

namespace enmf {

// Type codes for runtime dispatch.
enum : int { T_F64 = 0, T_F32 = 1, T_BF16 = 2, T_F16 = 3, T_CSR = 5 };

// X of the sparse form: the caller's compressed rows and the context's
// transpose (compressed columns, every column's entries in row order).  A
// launcher given xdt = T_CSR takes X as a pointer to this host struct.
// Work of one product (X B or X^T B): the rows cut into items of at most
// SPMM_SEG stored entries (at least one item per row, so empty rows are
// written).  An item of a row with one item writes the row of the output; the
// items of a longer row write partial rows to consecutive slots, summed in
// slot order by the fix-up (split rows: row, first slot, number of slots).
constexpr int SPMM_SEG = 2048;
struct SpmmPlan {
  int32_t* item_row;        // nitems
  int64_t* item_p;          // 2 nitems: first and one-past-last entry
  int32_t* item_slot;       // nitems: partial slot, or -1 (writes the output row)
  int64_t nitems;
  int32_t* split_row;       // nsplit
  int32_t* split_base;      // nsplit
  int32_t* split_cnt;       // nsplit
  int64_t nsplit;
  void* partial;            // slots x LMAX of the factors' type
};
struct CsrX {
  const int64_t* row_ptr;   // m + 1
  const int32_t* col;       // nnz
  const void* val;          // nnz, vdt
  int64_t* col_ptr;         // n + 1
  int32_t* row_t;           // nnz
  void* val_t;              // nnz, vdt
  int64_t m, n, nnz;
  int vdt;                  // T_F64 or T_F32 (the factors' type)
  SpmmPlan plan[2];         // X B, X^T B
};
// Bounds of a plan's arrays for `rows` rows and nnz entries.
inline int64_t spmm_max_items(int64_t rows, int64_t nnz) { return rows + nnz / SPMM_SEG + 1; }
inline int64_t spmm_max_split(int64_t nnz) { return nnz / (SPMM_SEG + 1) + 1; }
inline int64_t spmm_max_slots(int64_t nnz) { return 2 * (nnz / SPMM_SEG) + 2; }
void launch_csr_check(const CsrX& x, int* err, cudaStream_t s);
// out[e] = in[e] converted (FP32 <-> FP64), e < count
void launch_cast(const void* in, int in_dt, void* out, int out_dt, int64_t count, cudaStream_t s);
size_t csr_transpose_scratch(int64_t m, int64_t n, int64_t* nblk_out, int64_t* rows_per_blk_out);
void launch_csr_transpose(const CsrX& x, void* scratch, int64_t* col_ptr, int32_t* row_t,
                          void* val_t, cudaStream_t s);
// C = X B (trans = false) or X^T B (trans = true); B and C of type fdt.
void launch_spmm(const CsrX& x, bool trans, const void* B, int ldb, int k, void* C, int ldc,
                 int fdt, int num_sms, cudaStream_t s);
void launch_csr_normx2(const CsrX& x, double* part, double* out, int* err, cudaStream_t s);
// Fills pl's item and split arrays (device, sized by the spmm_max_* bounds)
// from the host copy of a product's row pointers; synchronises s.
bool build_spmm_plan(const int64_t* rp, int64_t rows, SpmmPlan& pl, cudaStream_t s);



inline size_t type_size(int t) { return t == T_F64 ? 8 : t == T_F32 ? 4 : 2; }

// Iteration state of Algorithm 3, resident in device memory so that the
// stage decision (ascent vs HALS) never needs a host round trip.
struct DevState {
  int stage;          // 0 ascent (Alg. 3 lines 5-11), 1 HALS (line 12)
  int k;              // alternations done
  int asc_iters;
  int hals_iters;
  int negU, negV;     // a negative entry remains after this half (ascent)
  int admm_done;
  int admm_steps;
  int svd_rank;
  int jac_sweeps;      // Jacobi sweeps of the last polar update (diagnostic)
  double s_u, s_v;            // shift steps of Eq. 8 / 9
  double maxneg_u, maxneg_v;  // max(-U), max(-V) when the stage started
  double normX2;              // ||X||_F^2
  double dR;                  // last ADMM ||R_k+1 - R_k||_F
  double rho;                 // ADMM penalty
  double negmass;             // sum h(.) scratch
  double svd_res;             // SVD start residual
  double sigma1;
  double f_last;              // objective after the last alternation
  GridBarrier bar;
};

// Number of fixed-order partial sums used by the reduction kernels.  It does
// not depend on the device, so results are reproducible across GPUs.
constexpr int NPART = 256;

// Host-side count of kernel launches (measurement only).
void note_launch(int n);

// Split-K choice for the SIMT sweeps (also used to size the workspace).
int choose_splits(int64_t rows_out, int64_t red_len, int k, int bm, int num_sms);
// Split-K count of the FP32-factor SIMT sweep (FP32 / 16-bit X).
int sweep_splits_f32(int64_t rows_out, int64_t red_len, int k, int num_sms);

// ---------------------------------------------------------------- sweep.cu
// C (rows_out x k, leading dim ldc) = X B (xv) or X^T B (xtu), FP64 or FP32
// accumulation by fdt; X element type xdt.  `part` is split-K scratch.
void launch_xv(const void* X, int xdt, int64_t m, int64_t n, int64_t ldx, const void* B, int ldb,
               int k, void* C, int ldc, int fdt, void* part, int num_sms, cudaStream_t s);
void launch_xtu(const void* X, int xdt, int64_t m, int64_t n, int64_t ldx, const void* B, int ldb,
                int k, void* C, int ldc, int fdt, void* part, int num_sms, cudaStream_t s);
// G (ka x kb, FP64, row-major) = A^T B over `rows` rows.
void launch_gram(const void* A, int lda, int ka, const void* B, int ldb, int kb, int64_t rows,
                 int fdt, double* part, double* G, cudaStream_t s);
// out[0] = sum_ij A_ij B_ij (FP64).
void launch_dot(const void* A, int lda, const void* B, int ldb, int k, int64_t rows, int fdt,
                double* part, double* out, cudaStream_t s);
// out[0] = ||X||_F^2, and ERR_DOMAIN if X has a negative/non-finite entry.
void launch_normx2(const void* X, int xdt, int64_t m, int64_t n, int64_t ldx, double* part,
                   double* out, int* err, cudaStream_t s);
// out[0] = ||X - U V^T||_F^2 formed entry by entry.
void launch_residual_direct(const void* X, int xdt, int64_t m, int64_t n, int64_t ldx,
                            const void* U, const void* V, int r, int fdt, double* part,
                            double* out, cudaStream_t s);
// out[e] = sum over NPART blocks of part[b * width + e], in block order.
void launch_part_reduce(const double* part, int width, double* out, cudaStream_t s);
// Omega (rows x k, ld k) uniform(-1, 1) from (seed, i, j).
void launch_omega(void* F, int fdt, int64_t rows, int k, uint64_t seed, cudaStream_t s);

// ----------------------------------------------------------------- rows.cu
// The tail of a HALS-stage half step left to the next kernel on the stream:
// the Gram of the updated factor summed from its per-block partials and, for
// the V-half, the end of the alternation (objective, trace, counters).  The
// half step writes every field (pending = 1 when it left its tail, 0 when it
// ran it itself); the next tensor-core sweep pass of the iteration, or the
// flush at the end of an enmf_iterate call, runs it (hstep.cu, tc_sweep.cu).
struct HalfTail {
  const double* gpart;      // nb x kk block partials of the Gram
  double* G_out;            // kk
  const double* obj_part;   // nb: <U^T U, block partial> (V-half)
  const double* dot_part;   // nb: <A, F> (V-half)
  DevState* st;
  double* trace;
  int nb, kk, finalize, trace_idx;
  int pending;
};

struct HalfArgs {
  void* F;            // factor being updated (rows x k)
  const void* A;      // X V or X^T U for this half (rows x k, ld k)
  const double* G;    // Gram of the other factor (k x k)
  void* gbuf;         // PBCD gradient scratch (rows x k)
  unsigned long long* mask;  // PBCD mask bits (rows x 8 bytes)
  int64_t rows;
  int k;
  int fdt;
  int which;          // 0: U-half, 1: V-half
  int pbcd_max_iter;
  double eps;
  DevState* st;
  double* part;       // NPART x 2 scratch
  int* err;
  int* counts;        // PBCD sweep counts per ascent step (2 per step)
  int counts_cap;
  const void* dotA;   // if non-null: V-half also sums <dotA, F> into dot_part
  double* dot_part;
  // fused Gram of the updated factor: G_out (k x k, FP64) = F^T F, summed from
  // per-block partials gpart (grid x k x k) in block order after a grid barrier
  double* G_out;
  double* gpart;
  // fused end of the alternation (V-half): objective into trace[trace_idx]
  // from Gu (U^T U) and G_out (V^T V), then the stage update
  int finalize;
  const double* Gu;
  double* obj_part;   // per-block <Gu, Gram partial> (grid doubles)
  double* trace;
  int trace_idx;
  // gram_only: skip the row updates and only form G_out = F^T F with the same
  // block decomposition (so a Gram taken at the start of a call is bitwise the
  // one the previous call's last half-step produced)
  int gram_only;
  // FP32 factors, tensor-core sweeps: also write the updated F transposed as
  // a BF16 pair, th = bf16(F^T), tl = bf16(F^T - th) (k x ldt), the operand
  // of the next sweep (null: not written)
  void* th;
  void* tl;
  int64_t ldt;
  int t_f16;          // th / tl in FP16 (else BF16)
  // the grid barrier of the launch (&st->bar for one problem; one shared
  // barrier for every problem of a grouped launch)
  GridBarrier* bar;
  // A came from a one-problem tensor-core sweep run without fix-up: rows of
  // tiles cut by its stream-K ranges are the sum, in CTA order, of the
  // contributors' partial slots (cut_part: [G][2][128][cut_rp] floats, each
  // slot 128 rows x k flat) plus cut_corr; other rows are in A as is.
  // cut_part null: A is complete.
  const float* cut_part;
  const float* cut_corr;
  int64_t cut_W, cut_G;   // the sweep's work units and grid
  int cut_nkb, cut_rp;    // k-blocks per tile, slot row stride
  // A came from the fused kernel (fused.cu): row i is the sum over the
  // clusters q < sum_n, in cluster order, of sum_part[(q rows + i) k + l],
  // plus cut_corr (the X_lo term) when given.  Null: not used.
  const float* sum_part;
  int sum_n;
  // non-null: in the HALS stage the Gram sum and the end of the alternation
  // are left to the next sweep through this tail (one-problem launches only)
  HalfTail* tail;
};
// hstep.cu: one cooperative launch per half step; grid <= half_step_grid().
// pdl = 1: launched as a programmatic dependent of the previous kernel on s
// (the blocks wait for its completion before any access).
void launch_half_step(const HalfArgs& a, int grid, cudaStream_t s, int pdl = 0);
// Runs tails[0..n) that are pending and clears them (one small launch).
void launch_half_tail_flush(HalfTail* tails, int n, int num_sms, cudaStream_t s);
int half_step_grid(int fdt, int k, int num_sms, int64_t rows);
// Grouped half steps of np problems with FP32 factors (HalfArgs in device
// memory, all with the same `bar`); problem p owns blocks bbeg[p] ..
// bbeg[p + 1] - 1 (bbeg: np + 1 ints in device memory), rank padded to kp
// for all.  Grid bbeg[np] <= half_group_capacity(kp).
void launch_half_group(const HalfArgs* probs, const int* bbeg, int np, int grid, int kp,
                       cudaStream_t s);
int half_group_capacity(int kp, int num_sms);
void launch_state_init(const void* U, const void* V, int64_t m, int64_t n, int k, int fdt,
                       int n_shift, DevState* st, double* part, cudaStream_t s);
// ADMM pass of Algorithm 1 over W = [U; V] (see rows.cu).
void launch_admm_pass(const void* U, const void* V, int64_t m, int64_t n, int k, int fdt,
                      const double* R, void* Z, void* Y, double rho, int first, DevState* st,
                      double* part, cudaStream_t s);
// out rows = in rows * T (k_in x k_out, FP64 row-major); in/out may not alias.
void launch_row_transform(const void* in, int ld_in, int k_in, void* out, int ld_out, int k_out,
                          int64_t rows, int fdt, const double* T, cudaStream_t s);
// In-place rows * R (k x k).
void launch_apply_square(void* F, int64_t rows, int k, int fdt, const double* R, cudaStream_t s);
// out[0] = sum h(F) over rows (negative mass), in FP64.
void launch_negmass(const void* F, int64_t rows, int k, int fdt, double* part, double* out,
                    int accumulate, cudaStream_t s);
// Column sums of the first k columns of F (rows x ld) into out (k doubles).
void launch_colsum(const void* F, int64_t rows, int ld, int k, int fdt, double* part, double* out,
                   cudaStream_t s);
// SVD-start residual: sum_i ||Y_i Wr - Q_i Ur S||^2 (see rows.cu).
void launch_rr_residual(const void* Y, int ldy, int ky, const void* Q, int ldq, int kq,
                        int64_t rows, int r, int fdt, const double* Wr, const double* UrS,
                        double* part, double* out, cudaStream_t s);
// KKT partial measures for one factor (see rows.cu); out gets 8 doubles.
void launch_kkt_rows(const void* F, const void* A, const double* G, int64_t rows, int k, int fdt,
                     double* part, double* out, cudaStream_t s);

// One problem of the FP32-factor ADMM rotation (admm.cu).
struct AdmmArgs {
  const float* U;
  const float* V;
  int64_t m, n;
  int k;
  double* R;       // k x k FP64, R_k in, R at exit out
  float* Z;        // (m + n) x k
  float* Y;        // (m + n) x k, zero at entry
  double rho;
  int max_iter;
  double tol;
  DevState* st;
  double* part;    // (the problem's blocks) x k x k FP64
  double* M;       // k x k FP64
  int* err;
};
// Blocks of a cooperative grouped ADMM grid at rank pad kp (all resident),
// and the blocks one problem of rows = m + n rows gets (its own launch's
// grid, launch_admm_f32).
int admm_group_capacity(int kp, int num_sms);
int admm_blocks(int kp, int64_t rows, int num_sms);
// np problems of rank pad kp in one cooperative grid of `grid` blocks:
// problem p on blocks bbeg[p] .. bbeg[p + 1] - 1 (device arrays), every grid
// barrier on `bar`; each problem's results are those of its own launch.
void launch_admm_group(const AdmmArgs* probs, const int* bbeg, int np, int grid, int kp,
                       GridBarrier* bar, cudaStream_t s);
// ----------------------------------------------------------------- admm.cu
// All steps of Algorithm 1 for FP32 factors in one cooperative launch: W =
// [U; V], R (k x k FP64) from R_0 in / final R out, Z, Y ((m + n) x k, Y zero
// at entry), part (>= NPART x k x k doubles), M (k x k).  Updates st->dR,
// admm_steps, admm_done, jac_sweeps.
void launch_admm_f32(const float* U, const float* V, int64_t m, int64_t n, int k, double* R,
                     float* Z, float* Y, double rho, int max_iter, double tol, DevState* st,
                     double* part, double* M, int* err, int num_sms, cudaStream_t s);

// -------------------------------------------------------------- general.cu
// Algorithm 4 (generalized rotation U* R1 Lambda R2), the whole loop: its
// workspace size and the run (U, V overwritten by U* R1 Lambda R2 and
// V* R1 Lambda^-1 R2; R1, lam, R2 device FP64 outputs).  Synchronises.
size_t general_ws_bytes(int64_t m, int64_t n, int k, int fdt);
enmf_status run_general_rotation(const void* U, const void* V, int64_t m, int64_t n, int k,
                                 int fdt, void* ws, double rho, int max_iter, double tol,
                                 double* R1_out, double* lam_out, double* R2_out, int* err,
                                 int* steps_out, double* change_out, bool* converged,
                                 cudaStream_t s);

// ---------------------------------------------------------------- small.cu
// R = polar(M) of a k x k M with warm start D (Np x Np), no loop bookkeeping.
void launch_polar_plain(const double* M, int k, double* R, double* D, int* err, cudaStream_t s);
// R_new = polar(sum of NPART partial M's); dR, convergence, ADMM step count.
void launch_polar(const double* M, int k, double* R, double* D, double tol,
                  DevState* st, int* err, cudaStream_t s);
// Orthonormalising map of a Gram G (k x k), applied by launch_row_orth:
// scaled Cholesky (T = L, Tx = D, 1 / diag(L), mode 1), or when G is
// numerically rank deficient the eigen map by one-sided Jacobi (eigenvalues
// > tau * lambda_1 kept, T = V_k diag(l^-1/2), unused columns zero, mode 0).
// Tx: 2 LMAX + 1 doubles.  Writes *kept.
void launch_eig_orth(const double* G, int k, double tau, double* T, double* Tx, int* kept, int* err,
                     cudaStream_t s);
// One orthonormalising transform of a group (launch_eig_orth's arguments).
struct EigOrthProb {
  const double* G;
  int k;
  double tau;
  double* T;
  double* Tx;
  int* kept;
  int* err;
};
// count transforms in one launch, one CTA each (probs in device memory,
// max_k >= every k), each with the arithmetic of its own launch_eig_orth.
void launch_eig_orth_group(const EigOrthProb* probs, int count, int max_k, cudaStream_t s);
// out = in mapped by eig_orth's (T, Tx) row by row (rows x k, leading
// dimensions ld_in / ld_out; in place is safe).
void launch_row_orth(const void* in, int ld_in, void* out, int ld_out, int k, int64_t rows, int fdt,
                     const double* T, const double* Tx, cudaStream_t s);
// SVD of the (k2 x k1) matrix R2^T given R2 = P (k2 x k1 row-major):
// R2^T = Ut S Wt^T, sorted descending.  Writes sigma (k1), Ut (k1 x k1),
// Wt (k2 x k1).  See small.cu for layouts.  fp32_only: FP32 Jacobi sweeps
// only (for FP32-accurate P), else FP32 sweeps finished in FP64.
void launch_rr_svd(const double* P, int k2, int k1, double* sigma, double* Ut, double* Wt,
                   int fp32_only, int* err, cudaStream_t s);
// One Rayleigh-Ritz SVD of a group (launch_rr_svd's arguments).
struct RrSvdProb {
  const double* P;
  int k2, k1;
  double* sigma;
  double* Ut;
  double* Wt;
  int fp32_only;
  int* err;
};
// count SVDs in one launch, one CTA each (probs in device memory; max_k2 and
// max_k1 bound every problem's k2 and k1), each with the arithmetic of its own
// launch_rr_svd.
void launch_rr_svd_group(const RrSvdProb* probs, int count, int max_k2, int max_k1,
                         cudaStream_t s);
// Final SVD-start transforms with the sign rule (see small.cu).
void launch_svd_finish(const double* sigma, const double* Ut, const double* Wt, int k1, int k2,
                       int r, const double* colsumQ, const double* colsumQ2, double* Tu,
                       double* Tv, double* sigma_out, cudaStream_t s);
void launch_rr_prep(const double* sigma, const double* Ut, const double* Wt, int k1, int k2,
                    int r, double* Wr, double* UrS, DevState* st, cudaStream_t s);
// ------------------------------------------------------------- tc_sweep.cu
// One problem of a (grouped) tensor-core sweep, in device memory.  The sweep's
// work is the concatenation over problems of each problem's (output tile,
// k-block) units; w_begin / t_begin are this problem's first unit and first
// tile in that order.  mode 0: out = X B (+ corr), rows_out = m, red = n;
// mode 1: out = X^T B (+ corr), rows_out = n, red = m.  Maps: X (box 64 x 128),
// B^T hi and lo (box 64 x rp).
struct alignas(64) SweepProb {
  unsigned char mapX[128];
  unsigned char mapBh[128];
  unsigned char mapBl[128];
  int64_t rows_out, red;
  int64_t w_begin, t_begin;
  float* out;
  const float* corr;
  int r;
  int f16;          // X and factor as FP16 (else BF16)
  int xq;           // X as e4m3 codes with per-tile exponents (the FP8 form)
  int ntj;          // FP8 form: column tiles of X (exponent row stride)
  const int* xexp;  // FP8 form: exponent k of each 128 x 128 tile of X
  int l2hint;       // X tiles' L2 policy: 0 normal, 1 evict_last (X_hi, read
                    // every alternation), 2 evict_first (X_lo, read rarely)
  const HalfTail* tail;   // the previous half step's tail, run by the epilogue
                          // warps while the first accumulator fills (or null)
};
// Fills the sizes of d (maps and pointers set by the caller) and returns its
// work units (tiles x k-blocks) and tiles through *units / *tiles.
void tc_prob_sizes(int mode, SweepProb* d, int64_t rows_out, int64_t red, int r, int64_t w_begin,
                   int64_t t_begin, int64_t* units, int64_t* tiles);
// Grouped sweep over np problems (descriptors in device memory, in work
// order), W units in all; part needs grid x 2 x 128 x rp floats, counters one
// int per tile of all problems (zero between launches).
// fixup = 0 (one problem only): tiles cut by the stream-K ranges are left as
// partial slots for the consumer (see CutTiles).
// xq = 1: the FP8-form kernel (every descriptor's X is e4m3 codes).
// stages: X stages of the shared-memory ring, 0 = as many as fit (2..8).
// pdl = 1: launched as a programmatic dependent of the previous kernel on s
// (the CTAs start while it runs and request their first X tiles; nothing else
// is read or written before it has completed).  Only where that kernel does
// not write X.
void launch_tc_group(int mode, int rp, const SweepProb* probs, int np, int64_t W, float* part,
                     int* counters, int num_sms, int* err, cudaStream_t s, int fixup = 1,
                     int xq = 0, int stages = 0, int pdl = 0);
int tc_group_grid(int64_t W, int num_sms);
// 2D BF16 tensor map (CUtensorMap, 128 bytes at `map`) over a row-major
// (rows x cols, ld) array, box box_cols x box_rows, 128-byte swizzle.
// f16 = TC_MAP_U8: one-byte elements (FP8 codes).
constexpr int TC_MAP_U8 = 2;
bool tc_make_map(void* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
                 int box_cols, int box_rows, int f16 = 0);
int tc_rank_pad(int r);
// CTAs of a one-problem sweep (<= num_sms); part needs grid x 2 x 128 x rp floats.
int tc_grid(int64_t rows_out, int64_t red, int mode, int num_sms);
// The 16-bit pairs (f16: FP16, else BF16).  split_x flags ERR_DOMAIN for a
// negative or non-finite X entry, or one beyond the FP16 range.
void launch_split_transpose(const float* F, int64_t rows, int r, void* hi, void* lo, int64_t ldt,
                            int f16, cudaStream_t s);
void launch_split_x(const float* X, int64_t m, int64_t n, int64_t ldx, void* xh, void* xl,
                    int64_t ldh, int f16, int* err, cudaStream_t s);
// FP8 form staging: e4m3 codes (m x ldq bytes), X_lo (BF16, m x ldh) and one
// exponent per 128 x 128 tile (row-major over tiles); ERR_DOMAIN for a
// negative or non-finite entry or one beyond 448 * 2^100.
void launch_quant_x(const float* X, int64_t m, int64_t n, int64_t ldx, void* xq, int64_t ldq,
                    void* xl, int64_t ldh, int* xexp, int* err, cudaStream_t s);
constexpr int TC_KB_XV = 128, TC_KB_XT = 128;

// ---------------------------------------------------------------- fused.cu
// The single-pass HALS U-half (fused.cu), in device memory.  X_hi and the V^T
// pair are read through TMA maps (X: box 64 x 128; V^T hi / lo: box 64 x rp).
struct alignas(64) FusedDesc {
  unsigned char mapX[128];
  unsigned char mapVh[128];
  unsigned char mapVl[128];
  int64_t m, n, ldm;
  int r, S, T, C, Q, npanels, f16;
  const double* Gv;   // V^T V (r x r)
  const float* cv;    // X_lo V (m x r) added to X V, or null
  float* U;           // m x r, updated in place
  void* uth;          // U^T pair written for the X_lo pass (rp x ldm, 16-bit)
  void* utl;
  float* xtu;         // Q x n x r: each cluster's X^T U partial
  double* gpart;      // (Q C) x r x r: each CTA's U^T U partial
  double* Gu;         // r x r: U^T U, summed by the last CTA
  int* counter;       // arrival counter, zero between launches
  int* err;
  // diagnostics: %globaltimer stamps per CTA and panel (null: none recorded);
  // slot (cta * (stamp_panels + 1) + panel) * 8 + event
  long long* stamps;
  int stamp_panels;
};
// Launch shape: clusters of C CTAs, slice width S = T x 128 columns, ring
// depth nst, Q clusters (ok = 0: the shape does not fit; use the two passes).
struct FusedPlan {
  int ok, C, S, T, nst, Q, npanels;
  size_t smem;
};
FusedPlan fused_plan(int64_t m, int64_t n, int rp);
cudaError_t launch_fused(const FusedDesc* fd, const FusedPlan& pl, int rp, cudaStream_t s);

// --------------------------------------------------- equivalence (App. F, H)
// small.cu: Z = G^-1 C and its SVD R1 Lambda R2^T, Zit = R1 Lambda^-1 R2^T.
void launch_equiv_svd(const double* G, const double* C, int k, double* R1, double* lam, double* R2,
                      double* Z, double* Zit, int* err, cudaStream_t s);
// small.cu: the permutation check of App. H from the three Grams.
void launch_perm_check(const double* GAA, const double* GBB, const double* GAB, int k, double eps,
                       double keep_frac, int* b_of_a, int* count, cudaStream_t s);
// rows.cu: out[0] = sum_i ||B_i - A_i T||^2 (FP64).
void launch_transform_residual(const void* A, const void* B, int64_t rows, int k, int fdt,
                               const double* T, double* part, double* out, cudaStream_t s);

// KKT finalisation: combine the two factors' partial measures.
void launch_kkt_final(const double* pu, const double* pv, double* out, cudaStream_t s);

// Matrix completion (nmc.cu): one half of a round of Algorithm eNMC on the
// rows of F (U: which = 0, or V: which = 1) with the per-row masked Grams G
// (rows x KP x KP) and right-hand sides A (rows x KP) already formed.
struct NmcArgs {
  void* F;                   // rows x k, updated in place
  void* gbuf;                // rows x k gradient scratch
  const void* G;             // rows x KP x KP
  const void* A;             // rows x KP
  unsigned long long* mask;  // rows (bit l: entry l in the mask M+)
  double* part;              // >= 2 NPART doubles
  GridBarrier* bar;
  int* err;
  DevState* st;              // s_u, s_v
  int* counts;               // PBCD sweeps per half, or NULL
  int counts_cap;
  int64_t rows;
  int k, fdt, which, round, pbcd_max_iter;
  double eps;
};
int nmc_rank_pad(int k);
// G, A of type gdt (T_F64, or the factors' type fdt)
void launch_nmc_gram(const int64_t* rp, const int32_t* ix, const void* val, int64_t rows,
                     const void* B, int k, int fdt, int gdt, void* G, void* A, int num_sms,
                     cudaStream_t s);
int nmc_pbcd_grid(int fdt, int k, int num_sms, int64_t rows);
void launch_nmc_pbcd(const NmcArgs& a, int grid, cudaStream_t s);
// G, A FP64
void launch_nmc_solve(const void* G, const void* A, int64_t rows, int k, double lam, void* F,
                      int fdt, int* err, int num_sms, cudaStream_t s);
// part: NPART doubles; *out = scale * (sum over the stored entries of
// (x - u_i . v_j)^2), scale a power of two
void launch_nmc_objective(const CsrX& x, const void* U, const void* V, int k, int fdt,
                          double scale, double* part, double* out, cudaStream_t s);

}  // namespace enmf
