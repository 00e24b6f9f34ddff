// The context behind the opaque enmf_ctx handle of include/enmf.h, shared by
// the translation units of the C ABI (api.cu, batch.cu).
#pragma once

#include "internal.h"

using namespace enmf;

struct enmf_ctx {
  enmf_problem p;
  cudaStream_t stream;
  int device;
  int num_sms;
  int fdt;                  // factor/accumulate type code
  int xdt;                  // X type code
  enmf_status poison;       // ENMF_OK unless poisoned
  bool state_valid;         // iteration state initialised
  int grid_u, grid_v;       // cooperative half-step grids
  // workspace
  void* ws;
  size_t ws_bytes;
  DevState* st;
  int* err;
  int* kept;
  int* counts;
  int counts_cap;
  void* M0; void* M1; void* M2;  // m x LMAX
  void* N0; void* N1; void* N2;  // n x LMAX
  void* Zb; void* Yb;            // (m + n) x r
  unsigned long long* mask;      // max(m, n)
  void* splitk;
  size_t splitk_bytes;
  double* part;                  // NPART * (LMAX^2 + 8)
  double* dot_part;              // 4096
  double* pb_part;               // 2 * 4096
  double* Gu; double* Gv; double* Msm; double* R;
  double* T1; double* T2; double* Ut; double* Wt; double* sig;
  double* T1x;   // eig_orth's companion of T1 (see launch_eig_orth)
  double* Tu; double* Tv; double* Wr; double* UrS; double* csQ; double* csQ2;
  double* scal;                  // 64 scratch scalars
  HalfTail* tails;               // the HALS half steps' deferred tails (U, V)
  // the sparse form: the bound compressed-row descriptor and the context's
  // transpose (in the workspace)
  CsrX sx;
  bool sx_bound;
  int nmc_rounds;           // rounds of Algorithm eNMC since the last reset
  int64_t* csc_ptr;
  int32_t* csc_row;
  void* csc_val;
  // host-data staging for enmf_solve
  void* hX; void* hU; void* hV;
  size_t hX_bytes;
  // tensor-core sweep descriptors (device, 8 slots) and their host copies:
  // 0/1 X V main / X_lo pass and 2/3 X^T U main / X_lo pass of the iteration,
  // 4..7 the same for enmf_sweep's caller buffers
  SweepProb* dprob;
  SweepProb hprob[8];
  // the iteration loop of enmf_iterate as a CUDA graph (captured on a private
  // stream, replayed while every argument of the call is unchanged)
  struct IterKey {
    const void* X;
    void* U;
    void* V;
    double* trace;
    int n_iter, pbcd_max_iter, n_shift, correct_every, prof_every;
    double eps;
    int it0;                // first alternation index of the captured range
    int exact_until;        // alternations before this index refresh X_lo every time
    int overlap;            // the enmf_set_overlap flags the graph was captured with
    bool operator==(const IterKey& o) const {
      return X == o.X && U == o.U && V == o.V && trace == o.trace && n_iter == o.n_iter &&
             pbcd_max_iter == o.pbcd_max_iter && n_shift == o.n_shift &&
             correct_every == o.correct_every && prof_every == o.prof_every && eps == o.eps &&
             it0 == o.it0 && exact_until == o.exact_until && overlap == o.overlap;
    }
  };
  // slot 0: the alternation loop with the two-pass sweeps (any stage);
  // slot 1: the fused single-pass loop (HALS stage, fused.cu)
  cudaStream_t cap_stream;
  cudaGraphExec_t iter_graph[2];
  IterKey iter_key[2];
  int iter_graph_kernels[2];   // kernel launches per replay
  int iter_graph_npev[2];      // profiling events recorded per replay
  bool no_graph;            // capture failed once: launch eagerly
  // programmatic dependent launches inside the captured loop (enmf_set_overlap):
  // bit 0 the sweeps after a half step, bit 1 the half steps after a sweep
  int overlap;
  bool capturing;           // the loop is being captured
  bool adj;                 // the last captured node is one of the loop's kernels
  // fused single-pass HALS alternation (fused.cu); fz_plan.ok = 0: not used
  FusedPlan fz_plan;
  int fz_enabled;           // enmf_set_fused (default 1)
  int l2_keep;              // L2 policy of X_hi tiles (1 evict_last; ENMF_L2_KEEP=0 for normal)
  bool hals_known;          // the device state is known to be in the HALS stage
  void* fzws;               // its buffers: descriptor, X^T U partials, Gram partials, counter
  FusedDesc* dfz;
  FusedDesc hfz;
  float* fz_xtu;
  double* fz_gpart;
  int* fz_counter;
  long long* fz_stamps;     // diagnostics (ENMF_FUSED_STAMPS set at creation), else null
  int fz_stamp_panels;
  // event timing of the X sweeps (enmf_profile)
  int prof_every;
  int npev;
  cudaEvent_t pev[2 * 256];
  double prof_ms;
  long long prof_n;
  // precision form (tensor-core sweeps on BF16 or FP16 X)
  int tc;
  int tf16;                 // the 16-bit type is FP16 (else BF16)
  int xq;                   // FP8 form: X_hi as e4m3 codes, per-tile exponents
  int* xexp;                // FP8 form: exponent of each 128 x 128 tile of X
  int64_t ldq;              // FP8 form: row stride of the codes (bytes)
  int rp;
  int64_t ldh, ldn, ldm;
  int sv, st_split;
  void* tcws;
  size_t tcws_bytes;
  const void* xh;                // X_hi (context-owned, or the caller's BF16 X)
  void* xl;                      // X_lo (context-owned; null for BF16 input)
  void* own_xh;
  void* vth; void* vtl;          // V^T as a BF16 pair (rp x ldn)
  void* uth; void* utl;          // U^T as a BF16 pair (rp x ldm)
  float* tcpart;                 // stream-K partial slots
  int* tccount;                  // per-tile arrival counters (after the slots)
  float* cv; float* cu;          // X_lo V, X_lo^T U (correction)
  const void* staged_src;        // X pointer the staged copy belongs to
  alignas(64) unsigned char maps[6][128];   // X_hi, X_lo, Vt hi/lo, Ut hi/lo
};

enum { MAP_XH = 0, MAP_XL = 1, MAP_VH = 2, MAP_VL = 3, MAP_UH = 4, MAP_UL = 5 };

constexpr int PROF_PAIRS = 256;

// The row-update arguments of one half step (U-half: which 0, V-half: 1).
HalfArgs ctx_half_args(enmf_ctx* ctx, int which, void* F, const void* A, const double* G,
                       int64_t rows, const enmf_iter_opts& o, bool dot, double* G_out,
                       const double* Gu, double* trace, int trace_idx);
// Start of an iteration call: state (re)initialisation when asked or never
// done, ||X||^2, and V^T V (plus V's BF16 pair in the tensor-core form).
void ctx_iter_prologue(enmf_ctx* ctx, const void* X, void* U, void* V, int n_shift, bool reset);
enmf_status ctx_check_launch(enmf_ctx* ctx);
enmf_status ctx_sync_status(enmf_ctx* ctx);
