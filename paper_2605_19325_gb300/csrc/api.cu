// C ABI of libenmf: context, workspace and the five calls of the eNMF path.
// Every step of the path runs in the kernels of sweep.cu, rows.cu, small.cu
// (and tc_sweep.cu for the tensor-core form); this file only checks
// arguments, carves the workspace and enqueues launches.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "ctx.h"


// Accumulate the recorded (start, stop) event pairs into the sweep totals.
static enmf_status prof_harvest(enmf_ctx* ctx) {
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    ctx->poison = ENMF_ECUDA;
    return ENMF_ECUDA;
  }
  for (int i = 0; i + 1 < ctx->npev; i += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->pev[i], ctx->pev[i + 1]) == cudaSuccess) {
      ctx->prof_ms += ms;
      ctx->prof_n += 1;
    } else {
      cudaGetLastError();   // an unusable pair is skipped, not reported as a fault
    }
  }
  ctx->npev = 0;
  return ENMF_OK;
}

static const char* kStatus[] = {"ok", "invalid argument", "X has a negative or non-finite entry",
                                "out of device memory", "CUDA error", "device wait timed out",
                                "did not converge", "context busy", "call out of order"};

extern "C" const char* enmf_status_string(enmf_status s) {
  int i = (int)s;
  return (i >= 0 && i <= 8) ? kStatus[i] : "unknown status";
}

extern "C" const char* enmf_version(void) { return "enmf-gb300 0.1"; }

// Tensor-core form?  BF16 or FP16 X, or e4m3 codes (FP8 form), in the sweeps.
static bool tc_form(const enmf_problem* p) {
  return p->stream_dtype == ENMF_BF16 || p->stream_dtype == ENMF_F16 ||
         p->stream_dtype == ENMF_E4M3;
}

static bool valid_problem(const enmf_problem* p) {
  if (!p) return false;
  if (p->m < 1 || p->n < 1) return false;
  if (p->r < 1 || p->r > ENMF_MAX_RANK || p->r > p->m || p->r > p->n) return false;
  if (p->x_dtype == ENMF_CSR) {
    // compressed rows: int32 column and row indices, FP32 or FP64 values
    if (p->stream_dtype != 0 && p->stream_dtype != ENMF_CSR) return false;
    if (p->m >= 0x7fffffffLL || p->n >= 0x7fffffffLL) return false;
    if (p->nnz < 0 || p->nnz >= 0x7fffffffLL || (double)p->nnz > (double)p->m * (double)p->n)
      return false;
    return p->f_dtype == ENMF_F64 || p->f_dtype == ENMF_F32;
  }
  if (p->ldx < p->n) return false;
  if (p->x_dtype < ENMF_F64 || p->x_dtype > ENMF_F16) return false;
  if (tc_form(p)) {
    if (p->f_dtype != ENMF_F32) return false;
    // F32 X (split into a 16-bit pair) or X already of the stream type
    if (p->x_dtype != ENMF_F32 && p->x_dtype != p->stream_dtype) return false;
    // the FP8 form is staged from F32 X only, one staging block per 128 x 128
    // tile (at most 65535 tile rows in the grid's y dimension)
    if (p->stream_dtype == ENMF_E4M3 && (p->m + 127) / 128 > 65535) return false;
    if (p->x_dtype != ENMF_F32 && (p->ldx % 8) != 0) return false;
    if (p->m > 0x7fffffffLL || p->n > 0x7fffffffLL) return false;
  } else if (p->stream_dtype != 0 && p->stream_dtype != p->x_dtype) {
    return false;
  }
  if (p->f_dtype == ENMF_F64) return p->x_dtype == ENMF_F64;
  return p->f_dtype == ENMF_F32;
}

// Tensor-core buffers of the precision form (a separate allocation).
struct TcPlan {
  int rp;
  int64_t ldh, ldn, ldm, ldq;
  int sv, st;          // split arguments for X V and X^T U
  size_t xh, xl, xs, vt, ut, part, cv, cu, desc, total;
};

static TcPlan tc_plan(const enmf_problem* p, int num_sms) {
  TcPlan t;
  memset(&t, 0, sizeof(t));
  if (!tc_form(p)) return t;
  const int64_t m = p->m, n = p->n;
  t.rp = tc_rank_pad(p->r);
  t.ldh = (n + 7) / 8 * 8;
  t.ldn = (n + 7) / 8 * 8;
  t.ldm = (m + 7) / 8 * 8;
  t.sv = tc_grid(m, n, 0, num_sms);
  t.st = tc_grid(n, m, 1, num_sms);
  t.ldq = (n + 15) / 16 * 16;
  if (p->stream_dtype == ENMF_E4M3) {
    // codes, X_lo in BF16, one int exponent per 128 x 128 tile
    t.xh = (size_t)m * t.ldq;
    t.xl = (size_t)m * t.ldh * 2;
    t.xs = (size_t)((m + 127) / 128) * ((n + 127) / 128) * 4;
  } else {
    t.xh = p->x_dtype == ENMF_F32 ? (size_t)m * t.ldh * 2 : 0;
    t.xl = t.xh;
    t.xs = 0;
  }
  t.vt = (size_t)t.rp * t.ldn * 2;
  t.ut = (size_t)t.rp * t.ldm * 2;
  // stream-K partial slots: grid x 2 x 128 rows x rp, and one arrival counter
  // per output tile (kept in the same buffer, after the slots)
  t.part = (size_t)(t.sv > t.st ? t.sv : t.st) * 2 * 128 * t.rp * 4 +
           (size_t)(((m > n ? m : n) + 127) / 128 + 1) * 4;
  t.cv = (size_t)m * p->r * 4;
  t.cu = (size_t)n * p->r * 4;
  t.desc = 8 * sizeof(SweepProb);
  auto a = [](size_t b) { return (b + 1023) & ~(size_t)1023; };
  t.total = a(t.xh) + a(t.xl) + a(t.xs) + 2 * a(t.vt) + 2 * a(t.ut) + a(t.part) + a(t.cv) +
            a(t.cu) + a(t.desc) + 1024;
  return t;
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Layout {
  size_t off[40];
  size_t total;
};

// Workspace plan; the order here defines the carving in enmf_create.
static size_t plan(const enmf_problem* p, int num_sms, size_t* splitk_out) {
  const size_t fs = p->f_dtype == ENMF_F64 ? 8 : 4;
  const int bm = p->f_dtype == ENMF_F64 ? 32 : 64;
  const size_t mm = (size_t)p->m, nn = (size_t)p->n, r = (size_t)p->r;
  // split-K scratch: the largest splits x rows x k over every width k used
  size_t sk = 256;
  for (int k = 1; k <= LMAX; ++k) {
    int sv = choose_splits(p->m, p->n, k, bm, num_sms);
    int st = choose_splits(p->n, p->m, k, bm, num_sms);
    if (fs == 4) {   // the FP32-factor sweep of FP32 / 16-bit X
      const int sv2 = sweep_splits_f32(p->m, p->n, k, num_sms), st2 = sweep_splits_f32(p->n, p->m, k, num_sms);
      if (sv2 > sv) sv = sv2;
      if (st2 > st) st = st2;
    }
    if (sv > 1 && (size_t)sv * mm * k * fs > sk) sk = (size_t)sv * mm * k * fs;
    if (st > 1 && (size_t)st * nn * k * fs > sk) sk = (size_t)st * nn * k * fs;
  }
  if (splitk_out) *splitk_out = sk;
  size_t t = 0;
  t += al256(sizeof(DevState)) + al256(64) + al256(8192 * sizeof(int));
  t += 3 * al256(mm * LMAX * fs) + 3 * al256(nn * LMAX * fs);
  t += 2 * al256((mm + nn) * r * fs);
  t += al256((mm > nn ? mm : nn) * 8);
  t += al256(sk);
  t += al256((size_t)NPART * (LMAX * LMAX + 8) * 8);
  t += al256(4096 * 8) + al256(2 * 4096 * 8);
  t += 9 * al256((size_t)LMAX * LMAX * 8) + 2 * al256((size_t)LMAX * RMAX * 8);
  t += 2 * al256((size_t)LMAX * RMAX * 8) + 3 * al256(LMAX * 8) + al256(64 * 8);
  t += al256(2 * sizeof(HalfTail));
  if (p->x_dtype == ENMF_CSR) {  // the transpose: column pointers, row indices, values
    t += al256((nn + 1) * 8) + al256((size_t)p->nnz * 4) + al256((size_t)p->nnz * fs);
    // the work plans of X B and X^T B (items, split rows, partial slots)
    for (int d = 0; d < 2; ++d) {
      const int64_t rows = d == 0 ? p->m : p->n;
      t += 2 * al256((size_t)spmm_max_items(rows, p->nnz) * 4) +
           al256((size_t)spmm_max_items(rows, p->nnz) * 16);
      t += 3 * al256((size_t)spmm_max_split(p->nnz) * 4);
      t += al256((size_t)spmm_max_slots(p->nnz) * LMAX * fs);
    }
  }
  return t;
}

extern "C" enmf_status enmf_workspace_size(const enmf_problem* p, size_t* bytes) {
  if (!valid_problem(p) || !bytes) return ENMF_EINVAL;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *bytes = plan(p, sms, nullptr) + tc_plan(p, sms).total;
  if (tc_form(p) && p->stream_dtype != ENMF_E4M3) {
    const FusedPlan fp = fused_plan(p->m, p->n, tc_rank_pad(p->r));
    if (fp.ok)
      *bytes += al256(sizeof(FusedDesc)) + al256((size_t)fp.Q * p->n * p->r * 4) +
                al256((size_t)fp.Q * fp.C * p->r * p->r * 8) + 256;
  }
  return ENMF_OK;
}

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) { ctx->poison = ENMF_ECUDA; return ENMF_ECUDA; } \
  } while (0)

static enmf_status check_launch(enmf_ctx* ctx) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->poison = ENMF_ECUDA;
    return ENMF_ECUDA;
  }
  return ENMF_OK;
}

// Synchronise and translate the device status word.
static enmf_status bind_x(enmf_ctx* ctx, const void* X, const void** xin);

static enmf_status sync_status(enmf_ctx* ctx, bool clear_notconv = true) {
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    ctx->poison = ENMF_ECUDA;
    return ENMF_ECUDA;
  }
  int err = 0;
  e = cudaMemcpy(&err, ctx->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    ctx->poison = ENMF_ECUDA;
    return ENMF_ECUDA;
  }
  if (err & ERR_TIMEOUT) {
    ctx->poison = ENMF_ETIMEOUT;
    return ENMF_ETIMEOUT;
  }
  if (err & (ERR_DOMAIN | ERR_NOTCONV | ERR_NONFINITE | ERR_FORMAT)) {
    int keep = 0;
    cudaMemcpy(ctx->err, &keep, sizeof(int), cudaMemcpyHostToDevice);
    if (err & ERR_FORMAT) return ENMF_EINVAL;
    if (err & ERR_DOMAIN) return ENMF_EDOMAIN;
    if ((err & ERR_NOTCONV) && clear_notconv) return ENMF_ENOTCONV;
  }
  return ENMF_OK;
}

extern "C" enmf_status enmf_create(const enmf_problem* p, void* stream, enmf_ctx** out) {
  if (!valid_problem(p) || !out) return ENMF_EINVAL;
  *out = nullptr;
  enmf_ctx* ctx = new (std::nothrow) enmf_ctx();
  if (!ctx) return ENMF_ENOMEM;
  memset(ctx, 0, sizeof(*ctx));
  ctx->p = *p;
  ctx->stream = (cudaStream_t)stream;
  ctx->fdt = p->f_dtype == ENMF_F64 ? T_F64 : T_F32;
  ctx->xdt = p->x_dtype;
  if (cudaGetDevice(&ctx->device) != cudaSuccess) { delete ctx; return ENMF_ECUDA; }
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  size_t sk = 0;
  ctx->ws_bytes = plan(p, ctx->num_sms, &sk);
  if (cudaMallocAsync(&ctx->ws, ctx->ws_bytes, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return ENMF_ENOMEM;
  }
  const size_t fs = type_size(ctx->fdt);
  const size_t mm = (size_t)p->m, nn = (size_t)p->n, r = (size_t)p->r;
  char* b = (char*)ctx->ws;
  auto take = [&](size_t bytes) { void* q = b; b += al256(bytes); return q; };
  ctx->st = (DevState*)take(sizeof(DevState));
  ctx->err = (int*)take(64);
  ctx->kept = ctx->err + 4;
  ctx->counts = (int*)take(8192 * sizeof(int));
  ctx->counts_cap = 8192;
  ctx->M0 = take(mm * LMAX * fs); ctx->M1 = take(mm * LMAX * fs); ctx->M2 = take(mm * LMAX * fs);
  ctx->N0 = take(nn * LMAX * fs); ctx->N1 = take(nn * LMAX * fs); ctx->N2 = take(nn * LMAX * fs);
  ctx->Zb = take((mm + nn) * r * fs);
  ctx->Yb = take((mm + nn) * r * fs);
  ctx->mask = (unsigned long long*)take((mm > nn ? mm : nn) * 8);
  ctx->splitk = take(sk);
  ctx->splitk_bytes = sk;
  ctx->part = (double*)take((size_t)NPART * (LMAX * LMAX + 8) * 8);
  ctx->dot_part = (double*)take(4096 * 8);
  ctx->pb_part = (double*)take(2 * 4096 * 8);
  ctx->Gu = (double*)take(LMAX * LMAX * 8);
  ctx->Gv = (double*)take(LMAX * LMAX * 8);
  ctx->Msm = (double*)take(LMAX * LMAX * 8);
  ctx->R = (double*)take(LMAX * LMAX * 8);
  ctx->T1 = (double*)take(LMAX * LMAX * 8);
  ctx->T2 = (double*)take(LMAX * LMAX * 8);
  ctx->Ut = (double*)take(LMAX * LMAX * 8);
  ctx->Wt = (double*)take(LMAX * LMAX * 8);
  ctx->T1x = (double*)take(LMAX * LMAX * 8);
  ctx->Tu = (double*)take(LMAX * RMAX * 8);
  ctx->Tv = (double*)take(LMAX * RMAX * 8);
  ctx->Wr = (double*)take(LMAX * RMAX * 8);
  ctx->UrS = (double*)take(LMAX * RMAX * 8);
  ctx->sig = (double*)take(LMAX * 8);
  ctx->csQ = (double*)take(LMAX * 8);
  ctx->csQ2 = (double*)take(LMAX * 8);
  ctx->scal = (double*)take(64 * 8);
  ctx->tails = (HalfTail*)take(2 * sizeof(HalfTail));
  cudaMemsetAsync(ctx->tails, 0, 2 * sizeof(HalfTail), ctx->stream);
  if (p->x_dtype == ENMF_CSR) {
    ctx->csc_ptr = (int64_t*)take((nn + 1) * 8);
    ctx->csc_row = (int32_t*)take((size_t)p->nnz * 4);
    ctx->csc_val = take((size_t)p->nnz * fs);
    for (int d = 0; d < 2; ++d) {
      SpmmPlan& pl = ctx->sx.plan[d];
      const int64_t rows = d == 0 ? p->m : p->n;
      const size_t ni = (size_t)spmm_max_items(rows, p->nnz) * 4;
      const size_t ns = (size_t)spmm_max_split(p->nnz) * 4;
      pl.item_row = (int32_t*)take(ni);
      pl.item_p = (int64_t*)take(ni * 4);
      pl.item_slot = (int32_t*)take(ni);
      pl.split_row = (int32_t*)take(ns);
      pl.split_base = (int32_t*)take(ns);
      pl.split_cnt = (int32_t*)take(ns);
      pl.partial = take((size_t)spmm_max_slots(p->nnz) * LMAX * fs);
      pl.nitems = 0;
      pl.nsplit = 0;
    }
  }
  if ((size_t)(b - (char*)ctx->ws) > ctx->ws_bytes) {
    cudaFreeAsync(ctx->ws, ctx->stream);
    delete ctx;
    return ENMF_EINVAL;
  }
  cudaMemsetAsync(ctx->ws, 0, ctx->ws_bytes, ctx->stream);
  ctx->grid_u = half_step_grid(ctx->fdt, p->r, ctx->num_sms, p->m);
  ctx->grid_v = half_step_grid(ctx->fdt, p->r, ctx->num_sms, p->n);
  // at most 256 blocks: the fused Gram keeps one k x k partial per block in
  // the NPART x (LMAX^2 + 8) partial buffer
  if (ctx->grid_u > 256) ctx->grid_u = 256;
  if (ctx->grid_v > 256) ctx->grid_v = 256;
  if (tc_form(p)) {
    const TcPlan t = tc_plan(p, ctx->num_sms);
    ctx->tc = 1;
    ctx->rp = t.rp;
    ctx->ldh = t.ldh;
    ctx->ldn = t.ldn;
    ctx->ldm = t.ldm;
    ctx->sv = t.sv;
    ctx->st_split = t.st;
    ctx->tcws_bytes = t.total;
    if (cudaMallocAsync(&ctx->tcws, t.total, ctx->stream) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeAsync(ctx->ws, ctx->stream);
      delete ctx;
      return ENMF_ENOMEM;
    }
    cudaMemsetAsync(ctx->tcws, 0, t.total, ctx->stream);
    char* q = (char*)(((uintptr_t)ctx->tcws + 1023) & ~(uintptr_t)1023);
    auto grab = [&](size_t bytes) { void* o = q; q += (bytes + 1023) & ~(size_t)1023; return o; };
    ctx->own_xh = t.xh ? grab(t.xh) : nullptr;
    ctx->xl = t.xl ? grab(t.xl) : nullptr;
    ctx->xexp = t.xs ? (int*)grab(t.xs) : nullptr;
    ctx->xq = p->stream_dtype == ENMF_E4M3;
    ctx->ldq = t.ldq;
    ctx->vth = grab(t.vt);
    ctx->vtl = grab(t.vt);
    ctx->uth = grab(t.ut);
    ctx->utl = grab(t.ut);
    ctx->tcpart = (float*)grab(t.part);
    ctx->tccount = (int*)(ctx->tcpart + (size_t)(t.sv > t.st ? t.sv : t.st) * 2 * 128 * t.rp);
    ctx->cv = (float*)grab(t.cv);
    ctx->cu = (float*)grab(t.cu);
    ctx->dprob = (SweepProb*)grab(t.desc);
    ctx->tf16 = p->stream_dtype == ENMF_F16;
    const int f16 = ctx->tf16;
    bool ok = tc_make_map(ctx->maps[MAP_VH], ctx->vth, t.rp, p->n, t.ldn, 64, t.rp, f16) &&
              tc_make_map(ctx->maps[MAP_VL], ctx->vtl, t.rp, p->n, t.ldn, 64, t.rp, f16) &&
              tc_make_map(ctx->maps[MAP_UH], ctx->uth, t.rp, p->m, t.ldm, 64, t.rp, f16) &&
              tc_make_map(ctx->maps[MAP_UL], ctx->utl, t.rp, p->m, t.ldm, 64, t.rp, f16);
    if (!ok) {
      cudaFreeAsync(ctx->tcws, ctx->stream);
      cudaFreeAsync(ctx->ws, ctx->stream);
      delete ctx;
      return ENMF_ECUDA;
    }
  }
  // the fused single-pass HALS alternation (fused.cu), when the shape fits
  if (ctx->tc && !ctx->xq) {
    const FusedPlan fp = fused_plan(p->m, p->n, ctx->rp);
    if (fp.ok) {
      const size_t xtu = (size_t)fp.Q * p->n * p->r * 4;
      const size_t gp = (size_t)fp.Q * fp.C * p->r * p->r * 8;
      const size_t bytes = al256(sizeof(FusedDesc)) + al256(xtu) + al256(gp) + 256;
      if (cudaMallocAsync(&ctx->fzws, bytes, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->tcws) cudaFreeAsync(ctx->tcws, ctx->stream);
        cudaFreeAsync(ctx->ws, ctx->stream);
        delete ctx;
        return ENMF_ENOMEM;
      }
      cudaMemsetAsync(ctx->fzws, 0, bytes, ctx->stream);
      char* f = (char*)ctx->fzws;
      ctx->dfz = (FusedDesc*)f;
      f += al256(sizeof(FusedDesc));
      ctx->fz_xtu = (float*)f;
      f += al256(xtu);
      ctx->fz_gpart = (double*)f;
      f += al256(gp);
      ctx->fz_counter = (int*)f;
      ctx->fz_plan = fp;
      if (getenv("ENMF_FUSED_STAMPS")) {
        ctx->fz_stamp_panels = 32;   // per CTA, recorded in shared memory
        const size_t sb = (size_t)fp.Q * fp.C * (ctx->fz_stamp_panels + 1) * 8 * 8;
        if (cudaMalloc(&ctx->fz_stamps, sb) != cudaSuccess) {
          cudaGetLastError();
          ctx->fz_stamps = nullptr;
        } else {
          cudaMemsetAsync(ctx->fz_stamps, 0, sb, ctx->stream);
        }
      }
    }
  }
  // The fused pass is built and checked but, on this GPU, slower than the two
  // passes at the measured shapes (its per-panel exchange across the cluster
  // is latency-bound): off unless enmf_set_fused asks for it.
  ctx->fz_enabled = 0;
  ctx->overlap = 1;   // (enmf_set_overlap: the measured best)
  {
    const char* e = getenv("ENMF_L2_KEEP");   // diagnostics: 0 = normal L2 policy for X_hi
    ctx->l2_keep = (e && atoi(e) == 0) ? 0 : 1;
  }
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    if (ctx->fzws) cudaFreeAsync(ctx->fzws, ctx->stream);
    if (ctx->tcws) cudaFreeAsync(ctx->tcws, ctx->stream);
    cudaFreeAsync(ctx->ws, ctx->stream);
    delete ctx;
    return ENMF_ECUDA;
  }
  *out = ctx;
  return ENMF_OK;
}

// ------------------------------------------------------ precision form
extern "C" enmf_status enmf_stage_x(enmf_ctx* ctx, const void* X) {
  if (!ctx || !X) return ENMF_EINVAL;
  if (ctx->poison) return ctx->poison;
  if (!ctx->tc) return ENMF_ESTATE;
  const enmf_problem& p = ctx->p;
  if (ctx->xq) {
    launch_quant_x((const float*)X, p.m, p.n, p.ldx, ctx->own_xh, ctx->ldq, ctx->xl, ctx->ldh,
                   ctx->xexp, ctx->err, ctx->stream);
    if (cudaGetLastError() != cudaSuccess) {
      ctx->poison = ENMF_ECUDA;
      return ENMF_ECUDA;
    }
    ctx->xh = ctx->own_xh;
    // codes: one 128 x 128 box per unit; X_lo: two 64-column BF16 boxes
    if (!tc_make_map(ctx->maps[MAP_XH], ctx->xh, p.m, p.n, ctx->ldq, 128, 128, TC_MAP_U8) ||
        !tc_make_map(ctx->maps[MAP_XL], ctx->xl, p.m, p.n, ctx->ldh, 64, 128, 0))
      return ENMF_ECUDA;
  } else if (p.x_dtype == ENMF_F32) {
    launch_split_x((const float*)X, p.m, p.n, p.ldx, ctx->own_xh, ctx->xl, ctx->ldh, ctx->tf16,
                   ctx->err,
                   ctx->stream);
    if (cudaGetLastError() != cudaSuccess) {
      ctx->poison = ENMF_ECUDA;
      return ENMF_ECUDA;
    }
    ctx->xh = ctx->own_xh;
    if (!tc_make_map(ctx->maps[MAP_XH], ctx->xh, p.m, p.n, ctx->ldh, 64, 128, ctx->tf16) ||
        !tc_make_map(ctx->maps[MAP_XL], ctx->xl, p.m, p.n, ctx->ldh, 64, 128, ctx->tf16))
      return ENMF_ECUDA;
  } else {
    if (((uintptr_t)X & 15) != 0) return ENMF_EINVAL;
    ctx->xh = X;
    if (!tc_make_map(ctx->maps[MAP_XH], X, p.m, p.n, p.ldx, 64, 128, ctx->tf16)) return ENMF_ECUDA;
  }
  ctx->staged_src = X;
  return ENMF_OK;
}

extern "C" void enmf_destroy(enmf_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  // the workspaces come from the stream-ordered allocator: freeing them does
  // not synchronise the device (a serving loop retires contexts while other
  // solves run)
  if (ctx->ws) cudaFreeAsync(ctx->ws, ctx->stream);
  if (ctx->hX) cudaFree(ctx->hX);
  if (ctx->hU) cudaFree(ctx->hU);
  if (ctx->hV) cudaFree(ctx->hV);
  if (ctx->tcws) cudaFreeAsync(ctx->tcws, ctx->stream);
  if (ctx->prof_every >= 0 && ctx->pev[0])
    for (int i = 0; i < 2 * PROF_PAIRS; ++i) cudaEventDestroy(ctx->pev[i]);
  for (int g = 0; g < 2; ++g)
    if (ctx->iter_graph[g]) cudaGraphExecDestroy(ctx->iter_graph[g]);
  if (ctx->fzws) cudaFreeAsync(ctx->fzws, ctx->stream);
  if (ctx->fz_stamps) cudaFree(ctx->fz_stamps);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

#define GUARD(ctx)                           \
  do {                                       \
    if (!(ctx)) return ENMF_EINVAL;          \
    if ((ctx)->poison) return (ctx)->poison; \
  } while (0)

// ------------------------------------------------------------ orthonormalise
// F (rows x k, ld LMAX) -> orthonormal columns spanning its range, through
// `tmp`: two passes of the Gram eigen map (numerical-rank truncation).
static void orth2(enmf_ctx* ctx, void* F, void* tmp, int64_t rows, int k) {
  const double tau = ctx->fdt == T_F64 ? 1e-13 : 1e-11;
  cudaStream_t s = ctx->stream;
  launch_gram(F, LMAX, k, F, LMAX, k, rows, ctx->fdt, ctx->part, ctx->Gu, s);
  launch_eig_orth(ctx->Gu, k, tau, ctx->T1, ctx->T1x, ctx->kept, ctx->err, s);
  launch_row_orth(F, LMAX, tmp, LMAX, k, rows, ctx->fdt, ctx->T1, ctx->T1x, s);
  launch_gram(tmp, LMAX, k, tmp, LMAX, k, rows, ctx->fdt, ctx->part, ctx->Gu, s);
  launch_eig_orth(ctx->Gu, k, tau, ctx->T1, ctx->T1x, ctx->kept, ctx->err, s);
  launch_row_orth(tmp, LMAX, F, LMAX, k, rows, ctx->fdt, ctx->T1, ctx->T1x, s);
}

// ------------------------------------------------------------------ 1. SVD
// The SVD start in two parts, so that a group of contexts can share the
// FP64-finished Rayleigh-Ritz SVD launch (enmf_svd_init_group).  Part 1: the
// power iterations with their stopping test, leaving the last P (ctx->Msm)
// and its SVD (FP64-finished for FP64 factors, FP32 otherwise); *finish =
// whether the FP32-then-FP64 SVD of that P is still owed.
struct SvdRun {
  int l, it, r;
  double res, tol;
  bool finish;
};

static enmf_status svd_part1(enmf_ctx* ctx, const void*& X, const enmf_svd_opts* opts, SvdRun& sr) {
  {
    const void* xb = nullptr;
    const enmf_status brc = bind_x(ctx, X, &xb);
    if (brc) return brc;
    X = xb;
  }
  enmf_svd_opts o = {10, 40, ctx->fdt == T_F64 ? 1e-12 : 1e-5, 0x5eedull, 0};
  if (opts) {
    o = *opts;
    if (o.oversample < 0 || o.max_iters < 1 || !(o.tol >= 0)) return ENMF_EINVAL;
  }
  const enmf_problem& p = ctx->p;
  const int r = p.r;
  int l = r + o.oversample;
  if (l > LMAX) l = LMAX;
  if (l > p.m) l = (int)p.m;
  if (l > p.n) l = (int)p.n;
  cudaStream_t s = ctx->stream;
  const int fdt = ctx->fdt, xdt = ctx->xdt;
  const int64_t m = p.m, n = p.n;
  launch_normx2(X, xdt, m, n, p.ldx, ctx->part, &ctx->st->normX2, ctx->err, s);
  // Q = orth(X Omega)
  launch_omega(ctx->N0, fdt, n, LMAX, o.seed, s);
  launch_xv(X, xdt, m, n, p.ldx, ctx->N0, LMAX, l, ctx->M0, LMAX, fdt, ctx->splitk, ctx->num_sms, s);
  orth2(ctx, ctx->M0, ctx->M1, m, l);
  enmf_status rc = check_launch(ctx);
  if (rc) return rc;
  double res = INFINITY;
  int it = 0;
  for (; it < o.max_iters; ++it) {
    // Bt = X^T Q ; Q2 = orth(Bt) ; P = Q2^T Bt
    launch_xtu(X, xdt, m, n, p.ldx, ctx->M0, LMAX, l, ctx->N1, LMAX, fdt, ctx->splitk, ctx->num_sms, s);
    launch_gram(ctx->N1, LMAX, l, ctx->N1, LMAX, l, n, fdt, ctx->part, ctx->Gu, s);
    launch_eig_orth(ctx->Gu, l, fdt == T_F64 ? 1e-13 : 1e-11, ctx->T1, ctx->T1x, ctx->kept, ctx->err, s);
    launch_row_orth(ctx->N1, LMAX, ctx->N0, LMAX, l, n, fdt, ctx->T1, ctx->T1x, s);
    launch_gram(ctx->N0, LMAX, l, ctx->N0, LMAX, l, n, fdt, ctx->part, ctx->Gu, s);
    launch_eig_orth(ctx->Gu, l, fdt == T_F64 ? 1e-13 : 1e-11, ctx->T1, ctx->T1x, ctx->kept, ctx->err, s);
    launch_row_orth(ctx->N0, LMAX, ctx->N2, LMAX, l, n, fdt, ctx->T1, ctx->T1x, s);
    launch_gram(ctx->N2, LMAX, l, ctx->N1, LMAX, l, n, fdt, ctx->part, ctx->Msm, s);
    // with FP32 factors the stopping test below takes the FP32 Jacobi SVD
    // (its residual sits far below the FP32 tolerance); the start itself is
    // made from the FP64-finished SVD of the last P, after the loop, unless
    // opts->fp32_finish
    launch_rr_svd(ctx->Msm, l, l, ctx->sig, ctx->Ut, ctx->Wt, fdt == T_F32 ? 1 : 0, ctx->err, s);
    // Y = X Q2 (the next power iterate) and the residual ||Y W_r - Q U_r S_r||
    launch_xv(X, xdt, m, n, p.ldx, ctx->N2, LMAX, l, ctx->M1, LMAX, fdt, ctx->splitk, ctx->num_sms, s);
    launch_rr_prep(ctx->sig, ctx->Ut, ctx->Wt, l, l, r, ctx->Wr, ctx->UrS, ctx->st, s);
    launch_rr_residual(ctx->M1, LMAX, l, ctx->M0, LMAX, l, m, r, fdt, ctx->Wr, ctx->UrS,
                       ctx->part, &ctx->scal[0], s);
    rc = check_launch(ctx);
    if (rc) return rc;
    double hv[2];
    CK(cudaMemcpyAsync(&hv[0], &ctx->scal[0], sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&hv[1], &ctx->st->sigma1, sizeof(double), cudaMemcpyDeviceToHost, s));
    rc = sync_status(ctx, false);
    if (rc && rc != ENMF_ENOTCONV) return rc;
    res = hv[1] > 0 ? sqrt(hv[0]) / hv[1] : 0.0;
    if (res <= o.tol) { ++it; break; }
    if (it + 1 < o.max_iters) {
      // Q = orth(Y)
      launch_gram(ctx->M1, LMAX, l, ctx->M1, LMAX, l, m, fdt, ctx->part, ctx->Gu, s);
      launch_eig_orth(ctx->Gu, l, fdt == T_F64 ? 1e-13 : 1e-11, ctx->T1, ctx->T1x, ctx->kept, ctx->err, s);
      launch_row_orth(ctx->M1, LMAX, ctx->M2, LMAX, l, m, fdt, ctx->T1, ctx->T1x, s);
      launch_gram(ctx->M2, LMAX, l, ctx->M2, LMAX, l, m, fdt, ctx->part, ctx->Gu, s);
      launch_eig_orth(ctx->Gu, l, fdt == T_F64 ? 1e-13 : 1e-11, ctx->T1, ctx->T1x, ctx->kept, ctx->err, s);
      launch_row_orth(ctx->M2, LMAX, ctx->M0, LMAX, l, m, fdt, ctx->T1, ctx->T1x, s);
    }
  }
  sr.l = l;
  sr.it = it;
  sr.r = r;
  sr.res = res;
  sr.finish = fdt == T_F32 && !o.fp32_finish;
  sr.tol = o.tol;
  return ENMF_OK;
}

// Part 2: U* = Q Tu, V* = Q2 Tv with the sign rule, the rank kept, the status.
static enmf_status svd_part2(enmf_ctx* ctx, void* U, void* V, double* sigma, const SvdRun& sr,
                             enmf_svd_info* info) {
  const enmf_problem& p = ctx->p;
  cudaStream_t s = ctx->stream;
  const int fdt = ctx->fdt, l = sr.l, r = sr.r;
  const int64_t m = p.m, n = p.n;
  launch_colsum(ctx->M0, m, LMAX, l, fdt, ctx->part, ctx->csQ, s);
  launch_colsum(ctx->N2, n, LMAX, l, fdt, ctx->part, ctx->csQ2, s);
  launch_svd_finish(ctx->sig, ctx->Ut, ctx->Wt, l, l, r, ctx->csQ, ctx->csQ2, ctx->Tu, ctx->Tv,
                    sigma, s);
  launch_row_transform(ctx->M0, LMAX, l, U, r, r, m, fdt, ctx->Tu, s);
  launch_row_transform(ctx->N2, LMAX, l, V, r, r, n, fdt, ctx->Tv, s);
  enmf_status rc = check_launch(ctx);
  if (rc) return rc;
  int kept = l;
  CK(cudaMemcpyAsync(&kept, ctx->kept, sizeof(int), cudaMemcpyDeviceToHost, s));
  rc = sync_status(ctx);
  if (info) {
    info->iters = sr.it;
    info->rank = kept;
    info->residual = sr.res;
  }
  ctx->state_valid = false;
  ctx->hals_known = false;
  if (rc) return rc;
  return sr.res <= sr.tol ? ENMF_OK : ENMF_ENOTCONV;
}

// ------------------------------------------------------------------ 1. SVD
extern "C" enmf_status enmf_svd_init(enmf_ctx* ctx, const void* X, void* U, void* V,
                                     double* sigma, const enmf_svd_opts* opts,
                                     enmf_svd_info* info) {
  GUARD(ctx);
  if (!X || !U || !V) return ENMF_EINVAL;
  SvdRun sr;
  enmf_status rc = svd_part1(ctx, X, opts, sr);
  if (rc) return rc;
  if (sr.finish)
    launch_rr_svd(ctx->Msm, sr.l, sr.l, ctx->sig, ctx->Ut, ctx->Wt, 0, ctx->err, ctx->stream);
  return svd_part2(ctx, U, V, sigma, sr, info);
}

// Part 1 for a group, in lockstep: every problem runs exactly the kernels of
// its own svd_part1 in the same order, but the single-CTA steps (the Gram
// eigen maps and the stopping test's Rayleigh-Ritz SVD) of all problems run
// in one launch each, and one synchronisation per power iteration serves all
// the stopping tests.  st[i] != ENMF_OK marks a problem that failed.
template <typename P>
static P* upload_group(const std::vector<P>& h, cudaStream_t s) {
  void* d = nullptr;
  if (h.empty() || cudaMallocAsync(&d, sizeof(P) * h.size(), s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (cudaMemcpyAsync(d, h.data(), sizeof(P) * h.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaFreeAsync(d, s);
    return nullptr;
  }
  return (P*)d;
}

static enmf_status svd_part1_group(enmf_ctx* const* ctxs, const void* const* Xin, int count,
                                   const enmf_svd_opts* opts, std::vector<SvdRun>& sr,
                                   std::vector<enmf_status>& st) {
  cudaStream_t s = ctxs[0]->stream;
  std::vector<const void*> X((size_t)count);
  std::vector<enmf_svd_opts> os((size_t)count);
  std::vector<int> live;
  for (int i = 0; i < count; ++i) {
    enmf_ctx* ctx = ctxs[i];
    X[i] = Xin[i];
    const void* xb = nullptr;
    st[i] = bind_x(ctx, X[i], &xb);
    if (st[i]) continue;
    X[i] = xb;
    enmf_svd_opts o = {10, 40, ctx->fdt == T_F64 ? 1e-12 : 1e-5, 0x5eedull, 0};
    if (opts) {
      o = *opts;
      if (o.oversample < 0 || o.max_iters < 1 || !(o.tol >= 0)) {
        st[i] = ENMF_EINVAL;
        continue;
      }
    }
    os[i] = o;
    const enmf_problem& p = ctx->p;
    int l = p.r + o.oversample;
    if (l > LMAX) l = LMAX;
    if (l > p.m) l = (int)p.m;
    if (l > p.n) l = (int)p.n;
    sr[i].l = l;
    sr[i].r = p.r;
    sr[i].it = 0;
    sr[i].res = INFINITY;
    sr[i].tol = o.tol;
    sr[i].finish = ctx->fdt == T_F32 && !o.fp32_finish;
    live.push_back(i);
  }
  auto tau = [&](int i) { return ctxs[i]->fdt == T_F64 ? 1e-13 : 1e-11; };
  auto eig_group = [&](const std::vector<int>& idx) {
    if (idx.empty()) return true;
    std::vector<EigOrthProb> h;
    int mk = 0;
    for (int i : idx) {
      enmf_ctx* c = ctxs[i];
      h.push_back(EigOrthProb{c->Gu, sr[i].l, tau(i), c->T1, c->T1x, c->kept, c->err});
      if (sr[i].l > mk) mk = sr[i].l;
    }
    EigOrthProb* d = upload_group(h, s);
    if (!d) return false;
    launch_eig_orth_group(d, (int)h.size(), mk, s);
    cudaFreeAsync(d, s);
    return true;
  };
  // in -> (Gram, eigen map) -> tmp -> (Gram, eigen map) -> out, per problem
  // the buffers sel(i) gives, as orth2 and the loop's orthonormalisations
  auto orth_two = [&](const std::vector<int>& idx, auto sel) {
    for (int i : idx) {
      enmf_ctx* c = ctxs[i];
      void *in, *tmp, *out;
      int64_t rows;
      sel(c, in, tmp, out, rows);
      launch_gram(in, LMAX, sr[i].l, in, LMAX, sr[i].l, rows, c->fdt, c->part, c->Gu, s);
    }
    if (!eig_group(idx)) return false;
    for (int i : idx) {
      enmf_ctx* c = ctxs[i];
      void *in, *tmp, *out;
      int64_t rows;
      sel(c, in, tmp, out, rows);
      launch_row_orth(in, LMAX, tmp, LMAX, sr[i].l, rows, c->fdt, c->T1, c->T1x, s);
      launch_gram(tmp, LMAX, sr[i].l, tmp, LMAX, sr[i].l, rows, c->fdt, c->part, c->Gu, s);
    }
    if (!eig_group(idx)) return false;
    for (int i : idx) {
      enmf_ctx* c = ctxs[i];
      void *in, *tmp, *out;
      int64_t rows;
      sel(c, in, tmp, out, rows);
      launch_row_orth(tmp, LMAX, out, LMAX, sr[i].l, rows, c->fdt, c->T1, c->T1x, s);
    }
    return true;
  };
  // Q = orth(X Omega)
  for (int i : live) {
    enmf_ctx* c = ctxs[i];
    const enmf_problem& p = c->p;
    launch_normx2(X[i], c->xdt, p.m, p.n, p.ldx, c->part, &c->st->normX2, c->err, s);
    launch_omega(c->N0, c->fdt, p.n, LMAX, os[i].seed, s);
    launch_xv(X[i], c->xdt, p.m, p.n, p.ldx, c->N0, LMAX, sr[i].l, c->M0, LMAX, c->fdt, c->splitk,
              c->num_sms, s);
  }
  if (!orth_two(live, [](enmf_ctx* c, void*& in, void*& tmp, void*& out, int64_t& rows) {
        in = c->M0; tmp = c->M1; out = c->M0; rows = c->p.m; }))
    return ENMF_ENOMEM;
  for (int i : live) {
    st[i] = check_launch(ctxs[i]);
  }
  std::vector<int> act;
  for (int i : live)
    if (!st[i]) act.push_back(i);
  while (!act.empty()) {
    // Bt = X^T Q ; Q2 = orth(Bt) ; P = Q2^T Bt
    for (int i : act) {
      enmf_ctx* c = ctxs[i];
      const enmf_problem& p = c->p;
      launch_xtu(X[i], c->xdt, p.m, p.n, p.ldx, c->M0, LMAX, sr[i].l, c->N1, LMAX, c->fdt, c->splitk,
                 c->num_sms, s);
    }
    if (!orth_two(act, [](enmf_ctx* c, void*& in, void*& tmp, void*& out, int64_t& rows) {
          in = c->N1; tmp = c->N0; out = c->N2; rows = c->p.n; }))
      return ENMF_ENOMEM;
    std::vector<RrSvdProb> h;
    int mk = 0;
    for (int i : act) {
      enmf_ctx* c = ctxs[i];
      const int l = sr[i].l;
      launch_gram(c->N2, LMAX, l, c->N1, LMAX, l, c->p.n, c->fdt, c->part, c->Msm, s);
      h.push_back(RrSvdProb{c->Msm, l, l, c->sig, c->Ut, c->Wt, c->fdt == T_F32 ? 1 : 0, c->err});
      if (l > mk) mk = l;
    }
    RrSvdProb* d = upload_group(h, s);
    if (!d) return ENMF_ENOMEM;
    launch_rr_svd_group(d, (int)h.size(), mk, mk, s);
    cudaFreeAsync(d, s);
    // Y = X Q2 (the next power iterate) and the residual ||Y W_r - Q U_r S_r||
    for (int i : act) {
      enmf_ctx* c = ctxs[i];
      const enmf_problem& p = c->p;
      const int l = sr[i].l, r = sr[i].r;
      launch_xv(X[i], c->xdt, p.m, p.n, p.ldx, c->N2, LMAX, l, c->M1, LMAX, c->fdt, c->splitk,
                c->num_sms, s);
      launch_rr_prep(c->sig, c->Ut, c->Wt, l, l, r, c->Wr, c->UrS, c->st, s);
      launch_rr_residual(c->M1, LMAX, l, c->M0, LMAX, l, p.m, r, c->fdt, c->Wr, c->UrS, c->part,
                         &c->scal[0], s);
    }
    std::vector<int> next, orth;
    for (int i : act) {
      enmf_ctx* c = ctxs[i];
      st[i] = check_launch(c);
      if (st[i]) continue;
      double hv[2];
      if (cudaMemcpyAsync(&hv[0], &c->scal[0], sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaMemcpyAsync(&hv[1], &c->st->sigma1, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
        c->poison = ENMF_ECUDA;
        st[i] = ENMF_ECUDA;
        continue;
      }
      const enmf_status rc = sync_status(c, false);
      if (rc && rc != ENMF_ENOTCONV) {
        st[i] = rc;
        continue;
      }
      sr[i].res = hv[1] > 0 ? sqrt(hv[0]) / hv[1] : 0.0;
      if (sr[i].res <= os[i].tol) {
        ++sr[i].it;
        continue;
      }
      if (sr[i].it + 1 < os[i].max_iters) orth.push_back(i);
      ++sr[i].it;
      if (sr[i].it < os[i].max_iters) next.push_back(i);
    }
    // Q = orth(Y)
    if (!orth.empty() &&
        !orth_two(orth, [](enmf_ctx* c, void*& in, void*& tmp, void*& out, int64_t& rows) {
          in = c->M1; tmp = c->M2; out = c->M0; rows = c->p.m; }))
      return ENMF_ENOMEM;
    act.swap(next);
  }
  return ENMF_OK;
}

extern "C" enmf_status enmf_svd_init_group(enmf_ctx* const* ctxs, const void* const* X,
                                           void* const* U, void* const* V, double* const* sigma,
                                           int32_t count, const enmf_svd_opts* opts,
                                           enmf_svd_info* infos, enmf_status* status) {
  if (!ctxs || !X || !U || !V || count < 1) return ENMF_EINVAL;
  if (!ctxs[0]) return ENMF_EINVAL;
  cudaStream_t s = ctxs[0]->stream;
  for (int i = 0; i < count; ++i) {
    enmf_ctx* ctx = ctxs[i];
    if (!ctx || !X[i] || !U[i] || !V[i]) return ENMF_EINVAL;
    if (ctx->poison) return ctx->poison;
    if (ctx->stream != s || ctx->device != ctxs[0]->device) return ENMF_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctx) return ENMF_EINVAL;
  }
  std::vector<SvdRun> sr((size_t)count);
  std::vector<enmf_status> st((size_t)count, ENMF_OK);
  const enmf_status grc = svd_part1_group(ctxs, X, count, opts, sr, st);
  if (grc) return grc;
  std::vector<RrSvdProb> hp;
  int mk = 0;
  for (int i = 0; i < count; ++i) {
    if (st[i] || !sr[i].finish) continue;
    enmf_ctx* ctx = ctxs[i];
    hp.push_back(RrSvdProb{ctx->Msm, sr[i].l, sr[i].l, ctx->sig, ctx->Ut, ctx->Wt, 0, ctx->err});
    if (sr[i].l > mk) mk = sr[i].l;
  }
  if (!hp.empty()) {
    void* d = nullptr;
    const size_t bytes = sizeof(RrSvdProb) * hp.size();
    if (cudaMallocAsync(&d, bytes, s) != cudaSuccess) {
      cudaGetLastError();
      return ENMF_ENOMEM;
    }
    if (cudaMemcpyAsync(d, hp.data(), bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      for (int i = 0; i < count; ++i) ctxs[i]->poison = ENMF_ECUDA;
      return ENMF_ECUDA;
    }
    launch_rr_svd_group((const RrSvdProb*)d, (int)hp.size(), mk, mk, s);
    cudaFreeAsync(d, s);
  }
  enmf_status first = ENMF_OK;
  for (int i = 0; i < count; ++i) {
    if (!st[i]) st[i] = svd_part2(ctxs[i], U[i], V[i], sigma ? sigma[i] : nullptr, sr[i],
                                  infos ? &infos[i] : nullptr);
    if (status) status[i] = st[i];
    if (st[i] && st[i] != ENMF_ENOTCONV && !first) first = st[i];
  }
  return first;
}

// ------------------------------------------------------------- 2. rotation
// R0 = I and the polar kernel's warm-start basis D = I (Np x Np, Np = k
// rounded up to even).
__global__ void rot_start_kernel(double* R, double* D, int k, DevState* st) {
  const int Np = k + (k & 1);
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) R[e] = (e / k == e % k) ? 1.0 : 0.0;
  for (int e = threadIdx.x; e < Np * Np; e += blockDim.x) D[e] = (e / Np == e % Np) ? 1.0 : 0.0;
  if (threadIdx.x == 0) {
    st->admm_done = 0;
    st->admm_steps = 0;
    st->dR = 0.0;
  }
}

extern "C" enmf_status enmf_rotate(enmf_ctx* ctx, void* U, void* V, double* Rout,
                                   const enmf_admm_opts* opts, enmf_rotate_info* info) {
  GUARD(ctx);
  if (!U || !V) return ENMF_EINVAL;
  enmf_admm_opts o = {0.0, 3.0, 200, 1e-12, 0};
  if (opts) {
    o = *opts;
    if (o.max_iter < 1 || !(o.tol >= 0) || (o.rho <= 0 && !(o.rho_scale > 0))) return ENMF_EINVAL;
  }
  const enmf_problem& p = ctx->p;
  const int k = p.r, fdt = ctx->fdt;
  const int64_t m = p.m, n = p.n;
  cudaStream_t s = ctx->stream;
  // the working factors: the caller's, or (FP32 factors, o.f64) FP64 copies
  // with FP64 Z and Y, from the stream-ordered allocator for this call
  void* Uw = U;
  void* Vw = V;
  void* Zw = ctx->Zb;
  void* Yw = ctx->Yb;
  int wdt = fdt;
  void* tmp = nullptr;
  if (fdt == T_F32 && o.f64) {
    const size_t wb = (size_t)(m + n) * k * 8;
    if (cudaMallocAsync(&tmp, 3 * wb, s) != cudaSuccess) {
      cudaGetLastError();
      return ENMF_ENOMEM;
    }
    Uw = tmp;
    Vw = (char*)tmp + (size_t)m * k * 8;
    Zw = (char*)tmp + wb;
    Yw = (char*)tmp + 2 * wb;
    wdt = T_F64;
    launch_cast(U, T_F32, Uw, T_F64, m * k, s);
    launch_cast(V, T_F32, Vw, T_F64, n * k, s);
  }
  // negative mass before and ||W||_F^2 for rho
  launch_negmass(Uw, m, k, wdt, ctx->part, &ctx->scal[1], 0, s);
  launch_negmass(Vw, n, k, wdt, ctx->part, &ctx->scal[1], 1, s);
  launch_dot(Uw, k, Uw, k, k, m, wdt, ctx->part, &ctx->scal[2], s);
  launch_dot(Vw, k, Vw, k, k, n, wdt, ctx->part, &ctx->scal[3], s);
  double hs[4];
  CK(cudaMemcpyAsync(hs, ctx->scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  enmf_status rc = sync_status(ctx);
  if (rc) {
    if (tmp) cudaFreeAsync(tmp, s);
    return rc;
  }
  double rho = o.rho;
  if (!(rho > 0)) {
    double rms = sqrt((hs[2] + hs[3]) / ((double)(m + n) * k));
    rho = rms > 0 ? o.rho_scale / rms : 1.0;
  }
  CK(cudaMemsetAsync(Yw, 0, (size_t)(m + n) * k * type_size(wdt), s));
  rot_start_kernel<<<1, 256, 0, s>>>(ctx->R, ctx->T2, k, ctx->st);
  note_launch(1);
  const int check_every = 16;
  if (wdt == T_F32) {
    // every ADMM step in one persistent kernel (admm.cu)
    launch_admm_f32((const float*)U, (const float*)V, m, n, k, ctx->R, (float*)ctx->Zb,
                    (float*)ctx->Yb, rho, o.max_iter, o.tol, ctx->st, ctx->part, ctx->Msm,
                    ctx->err, ctx->num_sms, s);
  }
  // FP64 factors: one ADMM pass, the fixed-order sum of M = W^T B and the
  // warm-started FP64 Jacobi polar factor per step
  for (int it = 0; wdt == T_F64 && it < o.max_iter; ++it) {
    launch_admm_pass(Uw, Vw, m, n, k, wdt, ctx->R, Zw, Yw, rho, it == 0, ctx->st,
                     ctx->part, s);
    launch_part_reduce(ctx->part, k * k, ctx->Msm, s);
    launch_polar(ctx->Msm, k, ctx->R, ctx->T2, o.tol, ctx->st, ctx->err, s);
    if ((it + 1) % check_every == 0 && it + 1 < o.max_iter) {
      rc = check_launch(ctx);
      int done = 0;
      if (!rc && (cudaMemcpyAsync(&done, &ctx->st->admm_done, sizeof(int), cudaMemcpyDeviceToHost,
                                  s) != cudaSuccess ||
                  cudaStreamSynchronize(s) != cudaSuccess)) {
        ctx->poison = ENMF_ECUDA;
        rc = ENMF_ECUDA;
      }
      if (rc) {
        if (tmp) cudaFreeAsync(tmp, s);
        return rc;
      }
      if (done) break;
    }
  }
  launch_apply_square(Uw, m, k, wdt, ctx->R, s);
  launch_apply_square(Vw, n, k, wdt, ctx->R, s);
  if (tmp) {   // U* R, V* R formed in FP64, rounded to FP32 once
    launch_cast(Uw, T_F64, U, T_F32, m * k, s);
    launch_cast(Vw, T_F64, V, T_F32, n * k, s);
    cudaFreeAsync(tmp, s);
  }
  launch_negmass(U, m, k, fdt, ctx->part, &ctx->scal[4], 0, s);
  launch_negmass(V, n, k, fdt, ctx->part, &ctx->scal[4], 1, s);
  if (Rout) CK(cudaMemcpyAsync(Rout, ctx->R, (size_t)k * k * sizeof(double), cudaMemcpyDeviceToDevice, s));
  rc = check_launch(ctx);
  if (rc) return rc;
  DevState hst;
  double nm_out = 0;
  CK(cudaMemcpyAsync(&hst, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&nm_out, &ctx->scal[4], sizeof(double), cudaMemcpyDeviceToHost, s));
  rc = sync_status(ctx);
  if (info) {
    info->steps = hst.admm_steps;
    info->converged = hst.admm_done;
    info->rho = rho;
    info->dR = hst.dR;
    info->neg_mass_in = hs[1];
    info->neg_mass_out = nm_out;
  }
  ctx->state_valid = false;
  ctx->hals_known = false;
  return rc;
}

extern "C" enmf_status enmf_rotate_group(enmf_ctx* const* ctxs, void* const* U, void* const* V,
                                         int32_t count, const enmf_admm_opts* opts,
                                         enmf_rotate_info* infos) {
  if (!ctxs || !U || !V || count < 1) return ENMF_EINVAL;
  enmf_admm_opts o = {0.0, 3.0, 200, 1e-12, 0};
  if (opts) {
    o = *opts;
    if (o.max_iter < 1 || !(o.tol >= 0) || (o.rho <= 0 && !(o.rho_scale > 0)) || o.f64)
      return ENMF_EINVAL;
  }
  if (!ctxs[0]) return ENMF_EINVAL;
  cudaStream_t s = ctxs[0]->stream;
  const int kp = tc_rank_pad(ctxs[0]->p.r);
  for (int i = 0; i < count; ++i) {
    enmf_ctx* ctx = ctxs[i];
    if (!ctx || !U[i] || !V[i]) return ENMF_EINVAL;
    if (ctx->poison) return ctx->poison;
    if (ctx->fdt != T_F32 || ctx->stream != s || ctx->device != ctxs[0]->device ||
        tc_rank_pad(ctx->p.r) != kp)
      return ENMF_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctx) return ENMF_EINVAL;
  }
  // a failed CUDA call poisons every context of the group
  auto fail = [&](cudaError_t e) {
    if (e == cudaSuccess) return false;
    for (int i = 0; i < count; ++i) ctxs[i]->poison = ENMF_ECUDA;
    return true;
  };
  // negative mass before and ||W||_F^2 for rho, all problems, one round trip
  for (int i = 0; i < count; ++i) {
    enmf_ctx* ctx = ctxs[i];
    const int64_t m = ctx->p.m, n = ctx->p.n;
    const int k = ctx->p.r;
    launch_negmass(U[i], m, k, T_F32, ctx->part, &ctx->scal[1], 0, s);
    launch_negmass(V[i], n, k, T_F32, ctx->part, &ctx->scal[1], 1, s);
    launch_dot(U[i], k, U[i], k, k, m, T_F32, ctx->part, &ctx->scal[2], s);
    launch_dot(V[i], k, V[i], k, k, n, T_F32, ctx->part, &ctx->scal[3], s);
  }
  for (int i = 0; i < count; ++i) {
    const enmf_status rc = check_launch(ctxs[i]);
    if (rc) return rc;
  }
  std::vector<double> hs((size_t)count * 4);
  for (int i = 0; i < count; ++i)
    if (fail(cudaMemcpyAsync(&hs[(size_t)i * 4], ctxs[i]->scal, 4 * sizeof(double),
                             cudaMemcpyDeviceToHost, s)))
      return ENMF_ECUDA;
  for (int i = 0; i < count; ++i) {
    const enmf_status rc = sync_status(ctxs[i]);
    if (rc) return rc;
  }
  // the problems' descriptors, packed into grids of at most `cap` blocks
  const int cap = admm_group_capacity(kp, ctxs[0]->num_sms);
  std::vector<AdmmArgs> hp((size_t)count);
  std::vector<int> nbk((size_t)count);
  std::vector<double> rhos((size_t)count);
  for (int i = 0; i < count; ++i) {
    enmf_ctx* ctx = ctxs[i];
    const int64_t m = ctx->p.m, n = ctx->p.n;
    const int k = ctx->p.r;
    double rho = o.rho;
    if (!(rho > 0)) {
      const double rms = sqrt((hs[(size_t)i * 4 + 2] + hs[(size_t)i * 4 + 3]) / ((double)(m + n) * k));
      rho = rms > 0 ? o.rho_scale / rms : 1.0;
    }
    rhos[i] = rho;
    if (fail(cudaMemsetAsync(ctx->Yb, 0, (size_t)(m + n) * k * sizeof(float), s)))
      return ENMF_ECUDA;
    rot_start_kernel<<<1, 256, 0, s>>>(ctx->R, ctx->T2, k, ctx->st);
    note_launch(1);
    hp[i] = AdmmArgs{(const float*)U[i], (const float*)V[i], m, n, k, ctx->R, (float*)ctx->Zb,
                     (float*)ctx->Yb, rho, o.max_iter, o.tol, ctx->st, ctx->part, ctx->Msm,
                     ctx->err};
    nbk[i] = admm_blocks(kp, m + n, ctx->num_sms);
  }
  // (a problem whose own grid exceeds a grouped grid's -- not the case on a
  // GB300, where both kernels keep the same occupancy -- runs alone through
  // launch_admm_f32: seg_np = 0 marks it)
  std::vector<int> hb;            // per grid: its problems' block offsets (np + 1 each)
  std::vector<int> seg_first, seg_np, seg_grid, seg_b;
  for (int i = 0; i < count;) {
    if (nbk[i] > cap) {
      seg_b.push_back((int)hb.size());
      seg_first.push_back(i);
      seg_np.push_back(0);
      seg_grid.push_back(0);
      ++i;
      continue;
    }
    int used = 0, j = i;
    seg_b.push_back((int)hb.size());
    while (j < count && nbk[j] <= cap && (j == i || used + nbk[j] <= cap)) {
      hb.push_back(used);
      used += nbk[j];
      ++j;
    }
    hb.push_back(used);
    seg_first.push_back(i);
    seg_np.push_back(j - i);
    seg_grid.push_back(used);
    i = j;
  }
  const size_t pbytes = sizeof(AdmmArgs) * (size_t)count;
  void* dbuf = nullptr;
  if (cudaMallocAsync(&dbuf, pbytes + sizeof(int) * hb.size(), s) != cudaSuccess) {
    cudaGetLastError();
    return ENMF_ENOMEM;
  }
  AdmmArgs* dp = (AdmmArgs*)dbuf;
  int* db = (int*)((char*)dbuf + pbytes);
  if (fail(cudaMemcpyAsync(dp, hp.data(), pbytes, cudaMemcpyHostToDevice, s)) ||
      fail(cudaMemcpyAsync(db, hb.data(), sizeof(int) * hb.size(), cudaMemcpyHostToDevice, s)))
    return ENMF_ECUDA;
  for (size_t g = 0; g < seg_first.size(); ++g) {
    if (seg_np[g] == 0) {
      const AdmmArgs& a = hp[seg_first[g]];
      launch_admm_f32(a.U, a.V, a.m, a.n, a.k, a.R, a.Z, a.Y, a.rho, a.max_iter, a.tol, a.st,
                      a.part, a.M, a.err, ctxs[seg_first[g]]->num_sms, s);
      continue;
    }
    launch_admm_group(dp + seg_first[g], db + seg_b[g], seg_np[g], seg_grid[g], kp,
                      &ctxs[seg_first[g]]->st->bar, s);
  }
  cudaFreeAsync(dbuf, s);
  // U* R, V* R and the negative mass after
  for (int i = 0; i < count; ++i) {
    enmf_ctx* ctx = ctxs[i];
    const int64_t m = ctx->p.m, n = ctx->p.n;
    const int k = ctx->p.r;
    launch_apply_square(U[i], m, k, T_F32, ctx->R, s);
    launch_apply_square(V[i], n, k, T_F32, ctx->R, s);
    launch_negmass(U[i], m, k, T_F32, ctx->part, &ctx->scal[4], 0, s);
    launch_negmass(V[i], n, k, T_F32, ctx->part, &ctx->scal[4], 1, s);
  }
  enmf_status first = ENMF_OK;
  for (int i = 0; i < count; ++i) {
    const enmf_status rc = check_launch(ctxs[i]);
    if (rc && !first) first = rc;
  }
  if (first) return first;
  for (int i = 0; i < count; ++i) {
    enmf_ctx* ctx = ctxs[i];
    const enmf_status rc = sync_status(ctx);
    ctx->state_valid = false;
    ctx->hals_known = false;
    if (rc && !first) first = rc;
    if (rc && rc != ENMF_ENOTCONV) continue;   // (ENOTCONV: results stand, as in enmf_rotate)
    if (infos) {
      DevState hst;
      double nm_out = 0;
      if (fail(cudaMemcpy(&hst, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost)) ||
          fail(cudaMemcpy(&nm_out, &ctx->scal[4], sizeof(double), cudaMemcpyDeviceToHost)))
        return ENMF_ECUDA;
      infos[i].steps = hst.admm_steps;
      infos[i].converged = hst.admm_done;
      infos[i].rho = rhos[i];
      infos[i].dR = hst.dR;
      infos[i].neg_mass_in = hs[(size_t)i * 4 + 1];
      infos[i].neg_mass_out = nm_out;
    }
  }
  return first;
}

// ------------------------------------------------------------ 3. iterate
// One half of an alternation: the row updates of F (U or V), the Gram of the
// new F into G_out and, for the V-half, the end-of-alternation bookkeeping.
HalfArgs ctx_half_args(enmf_ctx* ctx, int which, void* F, const void* A, const double* G,
                       int64_t rows, const enmf_iter_opts& o, bool dot, double* G_out,
                       const double* Gu, double* trace, int trace_idx) {
  HalfArgs a;
  memset(&a, 0, sizeof(a));
  a.F = F;
  a.A = A;
  a.G = G;
  a.gbuf = which == 0 ? ctx->M1 : ctx->N1;
  a.mask = ctx->mask;
  a.rows = rows;
  a.k = ctx->p.r;
  a.fdt = ctx->fdt;
  a.which = which;
  a.pbcd_max_iter = o.pbcd_max_iter;
  a.eps = o.eps;
  a.st = ctx->st;
  a.part = ctx->pb_part;
  a.err = ctx->err;
  a.counts = ctx->counts;
  a.counts_cap = ctx->counts_cap;
  a.dotA = dot ? A : nullptr;
  a.dot_part = dot ? ctx->dot_part : nullptr;
  a.G_out = G_out;
  a.gpart = ctx->part;
  a.finalize = which == 1 ? 1 : 0;
  a.Gu = Gu;
  a.obj_part = ctx->dot_part + 2048;
  a.trace = trace;
  a.trace_idx = trace_idx;
  a.bar = &ctx->st->bar;
  if (ctx->tc) {
    a.th = which == 0 ? ctx->uth : ctx->vth;
    a.tl = which == 0 ? ctx->utl : ctx->vtl;
    a.ldt = which == 0 ? ctx->ldm : ctx->ldn;
    a.t_f16 = ctx->tf16;
  }
  return a;
}

static int64_t tc_units(enmf_ctx* ctx, int mode);

// Programmatic dependent launch for the next kernel of the captured loop:
// only while capturing, with the flag `bit` of enmf_set_overlap set, and when
// the node before it is a kernel of the loop (no event, copy or graph start
// in between).  Every launch of the loop marks itself as such a node.
static int pdl_next(enmf_ctx* ctx, int bit) {
  const int on = (ctx->capturing && ctx->adj && (ctx->overlap & bit)) ? 1 : 0;
  ctx->adj = ctx->capturing;
  return on;
}

// The half steps of enmf_iterate: in the tensor-core form, A comes from a
// main sweep pass run without fix-up, so the half step assembles its cut
// tiles (HalfArgs::cut_part).
static void run_half(enmf_ctx* ctx, int which, void* F, const void* A, const double* G, int64_t rows,
                     const enmf_iter_opts& o, bool dot, double* G_out, const double* Gu,
                     double* trace, int trace_idx) {
  HalfArgs a = ctx_half_args(ctx, which, F, A, G, rows, o, dot, G_out, Gu, trace, trace_idx);
  if (ctx->tc) {
    const int mode = which;   // U-half reads X V (mode 0), V-half X^T U (mode 1)
    const int64_t red = mode == 0 ? ctx->p.n : ctx->p.m;
    a.cut_part = ctx->tcpart;
    a.cut_corr = ctx->xl ? (mode == 0 ? ctx->cv : ctx->cu) : nullptr;
    a.cut_W = tc_units(ctx, mode);
    a.cut_G = tc_group_grid(a.cut_W, ctx->num_sms);
    a.cut_nkb = (int)((red + (mode == 0 ? TC_KB_XV : TC_KB_XT) - 1) / (mode == 0 ? TC_KB_XV : TC_KB_XT));
    a.cut_rp = ctx->rp;
    // in the HALS stage the Gram sum and the end of the alternation run in the
    // next main sweep pass (slot 0 / 2), or in the flush after the loop
    a.tail = ctx->tails + which;
  }
  launch_half_step(a, which == 0 ? ctx->grid_u : ctx->grid_v, ctx->stream,
                   ctx->tc ? pdl_next(ctx, 2) : 0);
}

// ------------------------------------------------------------ the sweeps
// corr: 0 = X_hi only, 1 = add the stored X_lo term, 2 = refresh the X_lo
// term with the current factor first (tensor-core form; ignored otherwise).
// Descriptor slot `slot` of the one-problem tensor-core sweep (mode 0: X V,
// mode 1: X^T U; lo: the X_lo pass), uploaded to the device only when it
// changes -- so inside a captured iteration loop, where every slot was
// refreshed before the capture, nothing is copied.
static const SweepProb* tc_desc(enmf_ctx* ctx, int slot, int mode, bool lo, float* out,
                                const float* corr) {
  const enmf_problem& p = ctx->p;
  SweepProb d;
  memset(&d, 0, sizeof(d));
  // the iteration's main passes run the tail the previous half step left:
  // X V (slot 0) the V-half's, X^T U (slot 2) the U-half's
  if (slot == 0) d.tail = ctx->tails + 1;
  if (slot == 2) d.tail = ctx->tails + 0;
  memcpy(d.mapX, ctx->maps[lo ? MAP_XL : MAP_XH], sizeof(d.mapX));
  memcpy(d.mapBh, ctx->maps[mode == 0 ? MAP_VH : MAP_UH], sizeof(d.mapBh));
  memcpy(d.mapBl, ctx->maps[mode == 0 ? MAP_VL : MAP_UL], sizeof(d.mapBl));
  int64_t units, tiles;
  tc_prob_sizes(mode, &d, mode == 0 ? p.m : p.n, mode == 0 ? p.n : p.m, p.r, 0, 0, &units, &tiles);
  d.out = out;
  d.corr = corr;
  d.f16 = ctx->tf16;
  d.l2hint = lo ? 2 : ctx->l2_keep;
  if (ctx->xq && !lo) {
    d.xq = 1;
    d.ntj = (int)((p.n + 127) / 128);
    d.xexp = ctx->xexp;
  }
  if (memcmp(&d, &ctx->hprob[slot], sizeof(d)) != 0) {
    ctx->hprob[slot] = d;
    cudaMemcpyAsync(ctx->dprob + slot, &ctx->hprob[slot], sizeof(d), cudaMemcpyHostToDevice,
                    ctx->stream);
    ctx->adj = false;
  }
  return ctx->dprob + slot;
}

// Work units (tiles x k-blocks) of the one-problem sweep in `mode`.
static int64_t tc_units(enmf_ctx* ctx, int mode) {
  SweepProb d;
  int64_t units, tiles;
  tc_prob_sizes(mode, &d, mode == 0 ? ctx->p.m : ctx->p.n, mode == 0 ? ctx->p.n : ctx->p.m,
                ctx->p.r, 0, 0, &units, &tiles);
  return units;
}

// Profiling: with `rec`, CUDA events bracket the main X pass alone (not the
// factor split or the X_lo correction pass).
static void prof_mark(enmf_ctx* ctx, bool rec) {
  // (external: inside a captured graph the record is a real event node)
  if (rec) {
    cudaEventRecordWithFlags(ctx->pev[ctx->npev++], ctx->stream, cudaEventRecordExternal);
    ctx->adj = false;
  }
}


// split = false: the BF16 pair of the factor is already current (written by
// the half step that produced the factor).
// fixup = false: the main pass leaves its cut tiles to the consumer (the
// half step of enmf_iterate, through ctx_half_args(..., cut = true)).
static void sweep_xv(enmf_ctx* ctx, const void* X, const void* V, void* out, int corr,
                     bool rec = false, bool split = true, bool fixup = true) {
  const enmf_problem& p = ctx->p;
  cudaStream_t s = ctx->stream;
  const int r = p.r;
  if (!ctx->tc) {
    prof_mark(ctx, rec);
    launch_xv(X, ctx->xdt, p.m, p.n, p.ldx, V, r, r, out, r, ctx->fdt, ctx->splitk, ctx->num_sms, s);
    prof_mark(ctx, rec);
    return;
  }
  if (split)
    launch_split_transpose((const float*)V, p.n, r, ctx->vth, ctx->vtl, ctx->ldn, ctx->tf16, s);
  const int base = out == ctx->M0 ? 0 : 4;
  if (corr == 2 && ctx->xl) {
    const SweepProb* d = tc_desc(ctx, base + 1, 0, true, ctx->cv, nullptr);
    launch_tc_group(0, ctx->rp, d, 1, tc_units(ctx, 0), ctx->tcpart, ctx->tccount, ctx->num_sms,
                    ctx->err, s, 1, 0, 0, pdl_next(ctx, 1));
  }
  const SweepProb* d = tc_desc(ctx, base, 0, false, (float*)out,
                               (corr >= 1 && ctx->xl) ? ctx->cv : nullptr);
  prof_mark(ctx, rec);
  launch_tc_group(0, ctx->rp, d, 1, tc_units(ctx, 0), ctx->tcpart, ctx->tccount, ctx->num_sms,
                  ctx->err, s, fixup ? 1 : 0, ctx->xq, 0, pdl_next(ctx, 1));
  prof_mark(ctx, rec);
}

static void sweep_xtu(enmf_ctx* ctx, const void* X, const void* U, void* out, int corr,
                      bool rec = false, bool split = true, bool fixup = true) {
  const enmf_problem& p = ctx->p;
  cudaStream_t s = ctx->stream;
  const int r = p.r;
  if (!ctx->tc) {
    prof_mark(ctx, rec);
    launch_xtu(X, ctx->xdt, p.m, p.n, p.ldx, U, r, r, out, r, ctx->fdt, ctx->splitk, ctx->num_sms, s);
    prof_mark(ctx, rec);
    return;
  }
  if (split)
    launch_split_transpose((const float*)U, p.m, r, ctx->uth, ctx->utl, ctx->ldm, ctx->tf16, s);
  const int base = out == ctx->N0 ? 2 : 6;
  if (corr == 2 && ctx->xl) {
    const SweepProb* d = tc_desc(ctx, base + 1, 1, true, ctx->cu, nullptr);
    launch_tc_group(1, ctx->rp, d, 1, tc_units(ctx, 1), ctx->tcpart, ctx->tccount, ctx->num_sms,
                    ctx->err, s, 1, 0, 0, pdl_next(ctx, 1));
  }
  const SweepProb* d = tc_desc(ctx, base, 1, false, (float*)out,
                               (corr >= 1 && ctx->xl) ? ctx->cu : nullptr);
  prof_mark(ctx, rec);
  launch_tc_group(1, ctx->rp, d, 1, tc_units(ctx, 1), ctx->tcpart, ctx->tccount, ctx->num_sms,
                  ctx->err, s, fixup ? 1 : 0, ctx->xq, 0, pdl_next(ctx, 1));
  prof_mark(ctx, rec);
}

static enmf_status check_staged(enmf_ctx* ctx, const void* X) {
  if (ctx->tc && ctx->staged_src != X) return ENMF_ESTATE;
  return ENMF_OK;
}

// The X the launchers see.  Dense forms: X itself.  The sparse form: X is the
// caller's host enmf_csr; a descriptor with new array pointers is checked on
// the device and the context's transpose is built (the work buffer comes from
// the stream-ordered allocator); the launchers then get &ctx->sx.
static enmf_status bind_x(enmf_ctx* ctx, const void* X, const void** xin) {
  *xin = X;
  if (ctx->xdt != T_CSR) return ENMF_OK;
  const enmf_csr* d = (const enmf_csr*)X;
  const enmf_problem& p = ctx->p;
  if (!d->row_ptr || (p.nnz > 0 && (!d->col || !d->val))) return ENMF_EINVAL;
  if (ctx->sx_bound && ctx->sx.row_ptr == d->row_ptr && ctx->sx.col == d->col &&
      ctx->sx.val == d->val) {
    *xin = &ctx->sx;
    return ENMF_OK;
  }
  ctx->sx_bound = false;
  // graphs captured with the previous descriptor's arrays are stale
  for (int g = 0; g < 2; ++g)
    if (ctx->iter_graph[g]) {
      cudaGraphExecDestroy(ctx->iter_graph[g]);
      ctx->iter_graph[g] = nullptr;
    }
  CsrX& x = ctx->sx;
  x.row_ptr = d->row_ptr;
  x.col = d->col;
  x.val = d->val;
  x.col_ptr = ctx->csc_ptr;
  x.row_t = ctx->csc_row;
  x.val_t = ctx->csc_val;
  x.m = p.m;
  x.n = p.n;
  x.nnz = p.nnz;
  x.vdt = ctx->fdt;
  cudaStream_t s = ctx->stream;
  launch_csr_check(x, ctx->err, s);
  enmf_status rc = check_launch(ctx);
  if (rc) return rc;
  rc = sync_status(ctx);
  if (rc) return rc;
  void* scratch = nullptr;
  if (cudaMallocAsync(&scratch, csr_transpose_scratch(p.m, p.n, nullptr, nullptr), s) !=
      cudaSuccess) {
    cudaGetLastError();
    return ENMF_ENOMEM;
  }
  launch_csr_transpose(x, scratch, x.col_ptr, x.row_t, x.val_t, s);
  cudaFreeAsync(scratch, s);
  rc = check_launch(ctx);
  if (rc) return rc;
  rc = sync_status(ctx);
  if (rc) return rc;
  // the balanced work plans of both products, from host copies of the row
  // and column pointers
  for (int d = 0; d < 2; ++d) {
    const int64_t rows = d == 0 ? p.m : p.n;
    std::vector<int64_t> hp((size_t)rows + 1);
    CK(cudaMemcpy(hp.data(), d == 0 ? x.row_ptr : x.col_ptr, ((size_t)rows + 1) * 8,
                  cudaMemcpyDeviceToHost));
    if (!build_spmm_plan(hp.data(), rows, x.plan[d], s)) {
      ctx->poison = ENMF_ECUDA;
      return ENMF_ECUDA;
    }
  }
  ctx->sx_bound = true;
  *xin = &ctx->sx;
  return ENMF_OK;
}

// ------------------------------------------------------- state checkpoint
// Fixed host layout of the exported iteration state (ENMF_STATE_BYTES).
struct StateBlob {
  uint32_t magic, version;
  int64_t m, n;
  int32_t r, x_dtype, f_dtype, stream_dtype;
  int32_t stage, k, asc_iters, hals_iters, negU, negV;
  double s_u, s_v, maxneg_u, maxneg_v, f_last;
  unsigned char reserved_[ENMF_STATE_BYTES - 104];
};
static_assert(sizeof(StateBlob) == ENMF_STATE_BYTES, "state blob layout");
static constexpr uint32_t STATE_MAGIC = 0x534D4E45u;   // "ENMS"
static constexpr uint32_t STATE_VERSION = 1;

extern "C" enmf_status enmf_state_export(enmf_ctx* ctx, void* buf, size_t* bytes) {
  GUARD(ctx);
  if (!buf || !bytes || *bytes < sizeof(StateBlob)) {
    if (bytes) *bytes = sizeof(StateBlob);
    return ENMF_EINVAL;
  }
  if (!ctx->state_valid) return ENMF_ESTATE;
  DevState hst;
  CK(cudaMemcpyAsync(&hst, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream));
  enmf_status rc = sync_status(ctx);
  if (rc) return rc;
  StateBlob b;
  memset(&b, 0, sizeof(b));
  b.magic = STATE_MAGIC;
  b.version = STATE_VERSION;
  b.m = ctx->p.m;
  b.n = ctx->p.n;
  b.r = ctx->p.r;
  b.x_dtype = ctx->p.x_dtype;
  b.f_dtype = ctx->p.f_dtype;
  b.stream_dtype = ctx->p.stream_dtype;
  b.stage = hst.stage;
  b.k = hst.k;
  b.asc_iters = hst.asc_iters;
  b.hals_iters = hst.hals_iters;
  b.negU = hst.negU;
  b.negV = hst.negV;
  b.s_u = hst.s_u;
  b.s_v = hst.s_v;
  b.maxneg_u = hst.maxneg_u;
  b.maxneg_v = hst.maxneg_v;
  b.f_last = hst.f_last;
  memcpy(buf, &b, sizeof(b));
  *bytes = sizeof(b);
  return ENMF_OK;
}

extern "C" enmf_status enmf_state_import(enmf_ctx* ctx, const void* buf, size_t bytes) {
  GUARD(ctx);
  if (!buf || bytes < sizeof(StateBlob)) return ENMF_EINVAL;
  StateBlob b;
  memcpy(&b, buf, sizeof(b));
  const enmf_problem& p = ctx->p;
  if (b.magic != STATE_MAGIC || b.version != STATE_VERSION || b.m != p.m || b.n != p.n ||
      b.r != p.r || b.x_dtype != p.x_dtype || b.f_dtype != p.f_dtype ||
      b.stream_dtype != p.stream_dtype)
    return ENMF_EINVAL;
  if (b.stage < 0 || b.stage > 1 || b.k < 0) return ENMF_EINVAL;
  // counters consistent, flags boolean, shift steps and negative maxima finite
  // and nonnegative, objective finite: anything else is a corrupt buffer
  if (b.asc_iters < 0 || b.hals_iters < 0 || (int64_t)b.asc_iters + b.hals_iters > b.k)
    return ENMF_EINVAL;
  if ((b.negU != 0 && b.negU != 1) || (b.negV != 0 && b.negV != 1)) return ENMF_EINVAL;
  const double nonneg[4] = {b.s_u, b.s_v, b.maxneg_u, b.maxneg_v};
  for (double v : nonneg)
    if (!(v >= 0.0) || isinf(v)) return ENMF_EINVAL;
  if (!isfinite(b.f_last)) return ENMF_EINVAL;
  // the device state keeps its own grid barrier word and scratch scalars
  DevState hst;
  CK(cudaMemcpyAsync(&hst, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream));
  enmf_status rc = sync_status(ctx);
  if (rc) return rc;
  hst.stage = b.stage;
  hst.k = b.k;
  hst.asc_iters = b.asc_iters;
  hst.hals_iters = b.hals_iters;
  hst.negU = b.negU;
  hst.negV = b.negV;
  hst.s_u = b.s_u;
  hst.s_v = b.s_v;
  hst.maxneg_u = b.maxneg_u;
  hst.maxneg_v = b.maxneg_v;
  hst.f_last = b.f_last;
  CK(cudaMemcpyAsync(ctx->st, &hst, sizeof(DevState), cudaMemcpyHostToDevice, ctx->stream));
  rc = sync_status(ctx);
  if (rc) return rc;
  ctx->state_valid = true;
  ctx->hals_known = false;
  return ENMF_OK;
}

// The staged decomposition, copied out densely (inspection and tests).
extern "C" enmf_status enmf_stage_copy(enmf_ctx* ctx, void* hi, void* lo, int32_t* tile_exp) {
  GUARD(ctx);
  if (!ctx->tc || !ctx->staged_src) return ENMF_ESTATE;
  if ((lo && !ctx->xl) || (tile_exp && !ctx->xq)) return ENMF_EINVAL;
  const enmf_problem& p = ctx->p;
  cudaStream_t s = ctx->stream;
  if (hi) {
    const size_t es = ctx->xq ? 1 : 2;
    const int64_t ld = ctx->xh == ctx->own_xh ? (ctx->xq ? ctx->ldq : ctx->ldh) : p.ldx;
    CK(cudaMemcpy2DAsync(hi, (size_t)p.n * es, ctx->xh, (size_t)ld * es, (size_t)p.n * es,
                         (size_t)p.m, cudaMemcpyDefault, s));
  }
  if (lo)
    CK(cudaMemcpy2DAsync(lo, (size_t)p.n * 2, ctx->xl, (size_t)ctx->ldh * 2, (size_t)p.n * 2,
                         (size_t)p.m, cudaMemcpyDefault, s));
  if (tile_exp) {
    const size_t tiles = (size_t)((p.m + 127) / 128) * (size_t)((p.n + 127) / 128);
    CK(cudaMemcpyAsync(tile_exp, ctx->xexp, tiles * 4, cudaMemcpyDefault, s));
  }
  return sync_status(ctx);
}

extern "C" enmf_status enmf_sweep(enmf_ctx* ctx, const void* X, const void* U, const void* V,
                                  void* XV, void* XtU, int32_t exact) {
  GUARD(ctx);
  if (!X || (XV && !V) || (XtU && !U)) return ENMF_EINVAL;
  {
    const void* xb = nullptr;
    const enmf_status brc = bind_x(ctx, X, &xb);
    if (brc) return brc;
    X = xb;
  }
  enmf_status rc = check_staged(ctx, X);
  if (rc) return rc;
  if (XV) sweep_xv(ctx, X, V, XV, exact ? 2 : 0);
  if (XtU) sweep_xtu(ctx, X, U, XtU, exact ? 2 : 0);
  return check_launch(ctx);
}

// Runs the alternation loop as a CUDA graph: captured once on a private
// stream (the caller's stream may be the legacy default stream, which cannot
// be captured), instantiated, and replayed on the caller's stream while the
// key is unchanged.  Returns false (nothing enqueued) when graphs cannot be
// used, so the caller launches the loop directly.
template <typename Loop>
static bool replay_iteration(enmf_ctx* ctx, int slot, const enmf_ctx::IterKey& key, Loop&& loop) {
  if (ctx->no_graph || key.n_iter < 4) return false;
  if (!ctx->iter_graph[slot] || !(ctx->iter_key[slot] == key)) {
    if (ctx->iter_graph[slot]) {
      cudaGraphExecDestroy(ctx->iter_graph[slot]);
      ctx->iter_graph[slot] = nullptr;
    }
    if (!ctx->cap_stream &&
        cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      ctx->no_graph = true;
      return false;
    }
    cudaStream_t user = ctx->stream;
    const int npev0 = ctx->npev;
    const long long l0 = enmf_launch_count();
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal) ==
              cudaSuccess;
    if (ok) {
      ctx->stream = ctx->cap_stream;
      ctx->capturing = true;
      ctx->adj = false;
      loop();
      ctx->capturing = false;
      ctx->stream = user;
      ok = cudaStreamEndCapture(ctx->cap_stream, &g) == cudaSuccess && g;
    }
    const int kernels = (int)(enmf_launch_count() - l0);
    note_launch(-kernels);   // captured, not launched
    const int npev = ctx->npev - npev0;
    ctx->npev = npev0;
    cudaGraphExec_t exec = nullptr;
    if (ok) ok = cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
      cudaGetLastError();
      if (ctx->overlap) {
        // capture again without programmatic dependent launches (the flags
        // in effect read back through enmf_set_overlap)
        ctx->overlap = 0;
        enmf_ctx::IterKey k2 = key;
        k2.overlap = 0;
        return replay_iteration(ctx, slot, k2, loop);
      }
      ctx->no_graph = true;
      return false;
    }
    ctx->iter_graph[slot] = exec;
    ctx->iter_key[slot] = key;
    ctx->iter_graph_kernels[slot] = kernels;
    ctx->iter_graph_npev[slot] = npev;
  }
  if (cudaGraphLaunch(ctx->iter_graph[slot], ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    ctx->no_graph = true;
    return false;
  }
  note_launch(ctx->iter_graph_kernels[slot]);
  ctx->npev += ctx->iter_graph_npev[slot];
  return true;
}

void ctx_iter_prologue(enmf_ctx* ctx, const void* X, void* U, void* V, int n_shift, bool reset) {
  const enmf_problem& p = ctx->p;
  const int k = p.r, fdt = ctx->fdt;
  const int64_t m = p.m, n = p.n;
  cudaStream_t s = ctx->stream;
  if (reset || !ctx->state_valid) {
    launch_state_init(U, V, m, n, k, fdt, n_shift, ctx->st, ctx->part, s);
    ctx->state_valid = true;
  }
  launch_normx2(X, ctx->xdt, m, n, p.ldx, ctx->part, &ctx->st->normX2, ctx->err, s);
  // V^T V with the V-half kernel's own decomposition (bitwise equal to the
  // Gram the previous call ended with, so calls can be split freely)
  HalfArgs g;
  memset(&g, 0, sizeof(g));
  g.F = V;
  g.rows = n;
  g.k = k;
  g.fdt = fdt;
  g.which = 1;
  g.st = ctx->st;
  g.err = ctx->err;
  g.G = ctx->Gu;   // unused (read into shared memory only)
  g.G_out = ctx->Gv;
  g.gpart = ctx->part;
  g.gram_only = 1;
  g.bar = &ctx->st->bar;
  if (ctx->tc) {   // and the 16-bit pair of V for the first sweep
    g.th = ctx->vth;
    g.tl = ctx->vtl;
    g.ldt = ctx->ldn;
    g.t_f16 = ctx->tf16;
  }
  launch_half_step(g, ctx->grid_v, s);
}

enmf_status ctx_check_launch(enmf_ctx* ctx) { return check_launch(ctx); }
enmf_status ctx_sync_status(enmf_ctx* ctx) { return sync_status(ctx); }

extern "C" enmf_status enmf_iterate(enmf_ctx* ctx, const void* X, void* U, void* V,
                                    const enmf_iter_opts* opts, enmf_iter_info* info) {
  GUARD(ctx);
  if (!X || !U || !V) return ENMF_EINVAL;
  {
    const void* xb = nullptr;
    const enmf_status brc = bind_x(ctx, X, &xb);
    if (brc) return brc;
    X = xb;
  }
  enmf_iter_opts o = {0, 5, 1e-4, 3, nullptr, 0, 1, 10};
  if (opts) o = *opts;
  if (o.n_iter < 0 || o.pbcd_max_iter < 0 || !(o.eps >= 0) || o.n_shift < 1) return ENMF_EINVAL;
  if (o.correct_every < 1) o.correct_every = 10;
  const enmf_problem& p = ctx->p;
  const int64_t m = p.m, n = p.n;
  cudaStream_t s = ctx->stream;
  enmf_status rc = check_staged(ctx, X);
  if (rc) return rc;
  const bool fresh = o.reset != 0 || !ctx->state_valid;   // a new ascent stage starts
  ctx_iter_prologue(ctx, X, U, V, o.n_shift, o.reset != 0);
  if (ctx->tc) {
    // the iteration's sweep descriptors, current before any capture
    tc_desc(ctx, 0, 0, false, (float*)ctx->M0, ctx->xl ? ctx->cv : nullptr);
    tc_desc(ctx, 1, 0, true, ctx->cv, nullptr);
    tc_desc(ctx, 2, 1, false, (float*)ctx->N0, ctx->xl ? ctx->cu : nullptr);
    tc_desc(ctx, 3, 1, true, ctx->cu, nullptr);
  }
  // the alternations: everything on the device, nothing read back (except
  // the stage once, below)
  // From a reset the ascent stage ends within n_shift alternations (the worst
  // negative entry is nonnegative after n_shift shifts of max(-F) /
  // (n_shift - 1/2)).  In the precision forms those alternations run with the
  // X_lo term refreshed every time: the ascent stage decides which KKT point
  // the descent reaches, and it is the phase most sensitive to the rounding of
  // X (reading R28).
  const int pre = fresh ? (o.n_iter < o.n_shift ? o.n_iter : o.n_shift) : 0;
  const int exact_until = (ctx->tc && ctx->xl) ? pre : 0;
  auto general = [&](int it0, int it1) {
    for (int it = it0; it < it1; ++it) {
      // precision form: refresh the X_lo terms every correct_every alternations,
      // and in every alternation of a fresh ascent stage
      const int corr = (it < exact_until || it % o.correct_every == 0) ? 2 : 1;
      const bool rec = ctx->prof_every > 0 && it % ctx->prof_every == 0 && corr == 1 &&
                       ctx->npev + 4 <= 2 * PROF_PAIRS;
      sweep_xv(ctx, X, V, ctx->M0, corr, rec, false, false);
      run_half(ctx, 0, U, ctx->M0, ctx->Gv, m, o, false, ctx->Gu, nullptr, nullptr, 0);
      sweep_xtu(ctx, X, U, ctx->N0, corr, rec, false, false);
      run_half(ctx, 1, V, ctx->N0, ctx->Gu, n, o, true, ctx->Gv, ctx->Gu, o.trace, it);
    }
    // the last half step's deferred tail (ctx->stream: inside a capture, the
    // capture stream)
    if (ctx->tc && it1 > it0) launch_half_tail_flush(ctx->tails, 2, ctx->num_sms, ctx->stream);
  };
  // HALS stage, tensor-core form: one fused pass over X per alternation
  // (fused.cu) for the U-half and both products, then the V-half over the
  // clusters' X^T U partials; the X_lo passes of a correction alternation run
  // before (X_lo V) and after (X_lo^T U, with the new U) the fused pass.
  auto fused = [&](int it0, int it1) {
    const int rp = ctx->rp;
    // ctx->stream, read here: inside a capture it is the capture stream
    cudaStream_t fs = ctx->stream;
    for (int it = it0; it < it1; ++it) {
      const int corr = (it % o.correct_every == 0) ? 2 : 1;
      const bool rec = ctx->prof_every > 0 && it % ctx->prof_every == 0 && corr == 1 &&
                       ctx->npev + 2 <= 2 * PROF_PAIRS;
      if (corr == 2 && ctx->xl)
        launch_tc_group(0, rp, ctx->dprob + 1, 1, tc_units(ctx, 0), ctx->tcpart, ctx->tccount,
                        ctx->num_sms, ctx->err, fs);
      prof_mark(ctx, rec);
      launch_fused(ctx->dfz, ctx->fz_plan, rp, fs);
      prof_mark(ctx, rec);
      if (corr == 2 && ctx->xl)
        launch_tc_group(1, rp, ctx->dprob + 3, 1, tc_units(ctx, 1), ctx->tcpart, ctx->tccount,
                        ctx->num_sms, ctx->err, fs);
      HalfArgs a = ctx_half_args(ctx, 1, V, nullptr, ctx->Gu, n, o, true, ctx->Gv, ctx->Gu,
                                 o.trace, it);
      a.sum_part = ctx->fz_xtu;
      a.sum_n = ctx->fz_plan.Q;
      a.cut_corr = ctx->xl ? ctx->cu : nullptr;
      launch_half_step(a, ctx->grid_v, fs);
    }
  };
  auto run = [&](int slot, int it0, int it1) {
    if (it1 <= it0) return;
    enmf_ctx::IterKey key = {X, U, V, o.trace, it1 - it0, o.pbcd_max_iter, o.n_shift,
                             o.correct_every, ctx->prof_every, o.eps, it0,
                             it0 < exact_until ? exact_until : 0, ctx->overlap};
    auto body = [&]() {
      if (slot == 0) general(it0, it1);
      else fused(it0, it1);
    };
    if (!replay_iteration(ctx, slot, key, body)) body();
  };
  const bool fz_ok = ctx->tc && ctx->fz_plan.ok && ctx->fz_enabled && ctx->fzws;
  if (fresh) ctx->hals_known = false;
  int it = 0;
  if (exact_until > 0 && !(fz_ok && !ctx->hals_known)) {
    run(0, 0, exact_until);
    it = exact_until;
  }
  if (fz_ok && !ctx->hals_known && o.n_iter > 0) {
    // the ascent stage with the two-pass sweeps, then the stage read once
    run(0, 0, pre);
    rc = check_launch(ctx);
    if (rc) return rc;
    int stage = 0;
    CK(cudaMemcpyAsync(&stage, &ctx->st->stage, sizeof(int), cudaMemcpyDeviceToHost, s));
    rc = sync_status(ctx);
    if (rc) return rc;
    ctx->hals_known = stage == 1;
    it = pre;
  }
  if (fz_ok && ctx->hals_known && it < o.n_iter) {
    FusedDesc d;
    memset(&d, 0, sizeof(d));
    memcpy(d.mapX, ctx->maps[MAP_XH], sizeof(d.mapX));
    memcpy(d.mapVh, ctx->maps[MAP_VH], sizeof(d.mapVh));
    memcpy(d.mapVl, ctx->maps[MAP_VL], sizeof(d.mapVl));
    d.m = m;
    d.n = n;
    d.ldm = ctx->ldm;
    d.r = p.r;
    d.S = ctx->fz_plan.S;
    d.T = ctx->fz_plan.T;
    d.C = ctx->fz_plan.C;
    d.Q = ctx->fz_plan.Q;
    d.npanels = ctx->fz_plan.npanels;
    d.f16 = ctx->tf16;
    d.Gv = ctx->Gv;
    d.cv = ctx->xl ? ctx->cv : nullptr;
    d.U = (float*)U;
    d.uth = ctx->uth;
    d.utl = ctx->utl;
    d.xtu = ctx->fz_xtu;
    d.gpart = ctx->fz_gpart;
    d.Gu = ctx->Gu;
    d.counter = ctx->fz_counter;
    d.err = ctx->err;
    d.stamps = ctx->fz_stamps;
    d.stamp_panels = ctx->fz_stamp_panels;
    if (memcmp(&d, &ctx->hfz, sizeof(d)) != 0) {
      ctx->hfz = d;
      CK(cudaMemcpyAsync(ctx->dfz, &ctx->hfz, sizeof(d), cudaMemcpyHostToDevice, s));
    }
    run(1, it, o.n_iter);
  } else {
    run(0, it, o.n_iter);
  }
  rc = check_launch(ctx);
  if (rc) return rc;
  if (ctx->npev > 0) {
    rc = prof_harvest(ctx);
    if (rc) return rc;
  }
  if (o.sync_info || info) {
    DevState hst;
    CK(cudaMemcpyAsync(&hst, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    rc = sync_status(ctx);
    if (info) {
      info->iters = hst.k;
      info->asc_iters = hst.asc_iters;
      info->hals_iters = hst.hals_iters;
      info->stage = hst.stage;
      info->s_u = hst.s_u;
      info->s_v = hst.s_v;
    }
    return rc;
  }
  return ENMF_OK;
}

extern "C" enmf_status enmf_set_overlap(enmf_ctx* ctx, int32_t flags, int32_t* in_effect) {
  GUARD(ctx);
  if (flags >= 0) {
    if (flags > 3) return ENMF_EINVAL;
    ctx->overlap = flags;
  }
  if (in_effect) *in_effect = ctx->overlap;
  return ENMF_OK;
}

extern "C" enmf_status enmf_set_fused(enmf_ctx* ctx, int32_t on, int32_t* available) {
  GUARD(ctx);
  if (on != 0 && on != 1) return ENMF_EINVAL;
  ctx->fz_enabled = on;
  if (available) *available = (ctx->tc && ctx->fz_plan.ok && ctx->fzws) ? 1 : 0;
  return ENMF_OK;
}

// ---------------------------------------- generalized rotation (Algorithm 4)
extern "C" enmf_status enmf_rotate_general(enmf_ctx* ctx, void* U, void* V, double* R1,
                                           double* lam, double* R2, const enmf_admm_opts* opts,
                                           enmf_rotate_info* info) {
  GUARD(ctx);
  if (!U || !V || !R1 || !lam || !R2) return ENMF_EINVAL;
  enmf_admm_opts o = {0.0, 3.0, 200, 1e-12};
  if (opts) {
    o = *opts;
    if (o.max_iter < 1 || !(o.tol >= 0) || (o.rho <= 0 && !(o.rho_scale > 0))) return ENMF_EINVAL;
  }
  const enmf_problem& p = ctx->p;
  const int k = p.r, fdt = ctx->fdt;
  const int64_t m = p.m, n = p.n;
  cudaStream_t s = ctx->stream;
  launch_negmass(U, m, k, fdt, ctx->part, &ctx->scal[1], 0, s);
  launch_negmass(V, n, k, fdt, ctx->part, &ctx->scal[1], 1, s);
  launch_dot(U, k, U, k, k, m, fdt, ctx->part, &ctx->scal[2], s);
  launch_dot(V, k, V, k, k, n, fdt, ctx->part, &ctx->scal[3], s);
  double hs[4];
  CK(cudaMemcpyAsync(hs, ctx->scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  enmf_status rc = sync_status(ctx);
  if (rc) return rc;
  double rho = o.rho;
  if (!(rho > 0)) {
    const double rms = sqrt((hs[2] + hs[3]) / ((double)(m + n) * k));
    rho = rms > 0 ? o.rho_scale / rms : 1.0;
  }
  void* ws = nullptr;
  const size_t wb = general_ws_bytes(m, n, k, fdt);
  if (cudaMallocAsync(&ws, wb, s) != cudaSuccess) {
    cudaGetLastError();
    return ENMF_ENOMEM;
  }
  int steps = 0;
  double change = 0.0;
  bool conv = false;
  rc = run_general_rotation(U, V, m, n, k, fdt, ws, rho, o.max_iter, o.tol, R1, lam, R2, ctx->err,
                            &steps, &change, &conv, s);
  cudaFreeAsync(ws, s);
  if (rc) {
    ctx->poison = rc;
    return rc;
  }
  launch_negmass(U, m, k, fdt, ctx->part, &ctx->scal[4], 0, s);
  launch_negmass(V, n, k, fdt, ctx->part, &ctx->scal[4], 1, s);
  double nm_out = 0.0;
  CK(cudaMemcpyAsync(&nm_out, &ctx->scal[4], sizeof(double), cudaMemcpyDeviceToHost, s));
  rc = sync_status(ctx);
  if (info) {
    info->steps = steps;
    info->converged = conv ? 1 : 0;
    info->rho = rho;
    info->dR = change;
    info->neg_mass_in = hs[1];
    info->neg_mass_out = nm_out;
  }
  ctx->state_valid = false;
  ctx->hals_known = false;
  return rc;
}

// ------------------------------------------- equivalence tools (App. F, H)
extern "C" enmf_status enmf_equiv_transform(enmf_ctx* ctx, const void* Ue, const void* Ve,
                                            const void* Ua, const void* Va, double* R1,
                                            double* lam, double* R2, double* delta2) {
  GUARD(ctx);
  if (!Ue || !Ve || !Ua || !Va || !R1 || !lam || !R2 || !delta2) return ENMF_EINVAL;
  const enmf_problem& p = ctx->p;
  const int k = p.r, fdt = ctx->fdt;
  cudaStream_t s = ctx->stream;
  launch_gram(Ue, k, k, Ue, k, k, p.m, fdt, ctx->part, ctx->T1, s);   // G = U_e^T U_e
  launch_gram(Ue, k, k, Ua, k, k, p.m, fdt, ctx->part, ctx->Ut, s);   // C = U_e^T U_alg
  launch_equiv_svd(ctx->T1, ctx->Ut, k, R1, lam, R2, ctx->T2, ctx->Wt, ctx->err, s);
  // delta_u^2 = ||U_alg - U_e Z||^2, delta_v^2 = ||V_alg - V_e Zit||^2
  launch_transform_residual(Ue, Ua, p.m, k, fdt, ctx->T2, ctx->part, &ctx->scal[8], s);
  launch_transform_residual(Ve, Va, p.n, k, fdt, ctx->Wt, ctx->part, &ctx->scal[9], s);
  double h[2];
  CK(cudaMemcpyAsync(h, &ctx->scal[8], 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  enmf_status rc = sync_status(ctx);
  delta2[0] = sqrt(h[0] > 0.0 ? h[0] : 0.0);
  delta2[1] = sqrt(h[1] > 0.0 ? h[1] : 0.0);
  return rc;
}

extern "C" enmf_status enmf_perm_check(enmf_ctx* ctx, const void* UA, const void* UB, double eps,
                                       double keep_frac, int32_t* b_of_a, int32_t* kept) {
  GUARD(ctx);
  if (!UA || !UB || !b_of_a || !kept || !(eps >= 0.0) || !(keep_frac >= 0.0) || keep_frac > 1.0)
    return ENMF_EINVAL;
  const enmf_problem& p = ctx->p;
  const int k = p.r, fdt = ctx->fdt;
  cudaStream_t s = ctx->stream;
  launch_gram(UA, k, k, UA, k, k, p.m, fdt, ctx->part, ctx->T1, s);
  launch_gram(UB, k, k, UB, k, k, p.m, fdt, ctx->part, ctx->T2, s);
  launch_gram(UA, k, k, UB, k, k, p.m, fdt, ctx->part, ctx->Ut, s);
  launch_perm_check(ctx->T1, ctx->T2, ctx->Ut, k, eps, keep_frac, ctx->counts, ctx->counts + RMAX,
                    s);
  int h[RMAX + 1];
  CK(cudaMemcpyAsync(h, ctx->counts, (RMAX + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
  enmf_status rc = sync_status(ctx);
  if (rc) return rc;
  for (int i = 0; i < k; ++i) b_of_a[i] = h[i];
  *kept = h[RMAX];
  return ENMF_OK;
}

extern "C" enmf_status enmf_fused_shape(enmf_ctx* ctx, int32_t* shape) {
  GUARD(ctx);
  if (!shape) return ENMF_EINVAL;
  const FusedPlan& f = ctx->fz_plan;
  shape[0] = f.ok && ctx->fzws ? 1 : 0;
  shape[1] = f.C;
  shape[2] = f.Q;
  shape[3] = f.S;
  shape[4] = f.nst;
  shape[5] = (int32_t)(f.smem / 1024);
  return ENMF_OK;
}

extern "C" enmf_status enmf_fused_stamps(enmf_ctx* ctx, long long* out, int64_t cap,
                                         int64_t* count) {
  GUARD(ctx);
  if (!count) return ENMF_EINVAL;
  if (!ctx->fz_stamps) {
    *count = 0;
    return ENMF_OK;
  }
  const int64_t n = (int64_t)ctx->fz_plan.Q * ctx->fz_plan.C * (ctx->fz_stamp_panels + 1) * 8;
  *count = n;
  if (out && cap >= n) {
    CK(cudaMemcpyAsync(out, ctx->fz_stamps, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    return sync_status(ctx);
  }
  return ENMF_OK;
}

extern "C" enmf_status enmf_set_wait_limit(enmf_ctx* ctx, int64_t cycles) {
  GUARD(ctx);
  if (cycles < 0 || cycles > 4000000000LL) return ENMF_EINVAL;
  const unsigned int v = (unsigned int)cycles;
  CK(cudaMemcpyAsync(&ctx->st->bar.spin, &v, sizeof(v), cudaMemcpyHostToDevice, ctx->stream));
  return sync_status(ctx);
}

extern "C" enmf_status enmf_profile(enmf_ctx* ctx, int32_t every) {
  GUARD(ctx);
  if (every < 0) return ENMF_EINVAL;
  if (every > 0 && !ctx->pev[0]) {
    for (int i = 0; i < 2 * PROF_PAIRS; ++i)
      if (cudaEventCreate(&ctx->pev[i]) != cudaSuccess) return ENMF_ECUDA;
  }
  ctx->prof_every = every;
  ctx->npev = 0;
  return ENMF_OK;
}

extern "C" enmf_status enmf_profile_read(enmf_ctx* ctx, double* sweep_ms, int64_t* sweeps,
                                         int32_t reset) {
  GUARD(ctx);
  if (!sweep_ms || !sweeps) return ENMF_EINVAL;
  if (ctx->npev > 0) {
    enmf_status rc = prof_harvest(ctx);
    if (rc) return rc;
  }
  *sweep_ms = ctx->prof_ms;
  *sweeps = ctx->prof_n;
  if (reset) {
    ctx->prof_ms = 0.0;
    ctx->prof_n = 0;
  }
  return ENMF_OK;
}

extern "C" enmf_status enmf_pbcd_counts(enmf_ctx* ctx, int32_t* out, int32_t cap, int32_t* count) {
  GUARD(ctx);
  if (!out || !count || cap < 0) return ENMF_EINVAL;
  DevState hst;
  CK(cudaMemcpyAsync(&hst, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  int nasc = hst.asc_iters;
  int ncopy = 2 * nasc;
  if (ncopy > cap) ncopy = cap;
  if (ncopy > ctx->counts_cap) ncopy = ctx->counts_cap;
  if (ncopy > 0) CK(cudaMemcpy(out, ctx->counts, ncopy * sizeof(int), cudaMemcpyDeviceToHost));
  *count = nasc;
  return ENMF_OK;
}

// ------------------------------------------------------------ 4. residual
extern "C" enmf_status enmf_residual(enmf_ctx* ctx, const void* X, const void* U, const void* V,
                                     double* out3, int32_t direct) {
  GUARD(ctx);
  if (!X || !U || !V || !out3) return ENMF_EINVAL;
  {
    const void* xb = nullptr;
    const enmf_status brc = bind_x(ctx, X, &xb);
    if (brc) return brc;
    X = xb;
  }
  const enmf_problem& p = ctx->p;
  const int k = p.r, fdt = ctx->fdt, xdt = ctx->xdt;
  const int64_t m = p.m, n = p.n;
  cudaStream_t s = ctx->stream;
  launch_normx2(X, xdt, m, n, p.ldx, ctx->part, &ctx->scal[8], ctx->err, s);
  const bool dense_direct = direct && xdt != T_CSR;
  if (dense_direct) {
    launch_residual_direct(X, xdt, m, n, p.ldx, U, V, k, fdt, ctx->part, &ctx->scal[9], s);
  } else if (xdt == T_CSR) {
    // sparse: ||X||^2 - 2 <U, X V> + <U^T U, V^T V>, the cross term summed
    // entry by entry over the stored entries (X V row by row)
    launch_xv(X, xdt, m, n, p.ldx, V, k, k, ctx->M0, k, fdt, ctx->splitk, ctx->num_sms, s);
    launch_dot(ctx->M0, k, U, k, k, m, fdt, ctx->part, &ctx->scal[10], s);
    launch_gram(U, k, k, U, k, k, m, fdt, ctx->part, ctx->Gu, s);
    launch_gram(V, k, k, V, k, k, n, fdt, ctx->part, ctx->Gv, s);
    launch_dot(ctx->Gu, k, ctx->Gv, k, k, k, T_F64, ctx->part, &ctx->scal[11], s);
  } else {
    launch_xtu(X, xdt, m, n, p.ldx, U, k, k, ctx->N0, k, fdt, ctx->splitk, ctx->num_sms, s);
    launch_dot(ctx->N0, k, V, k, k, n, fdt, ctx->part, &ctx->scal[10], s);
    launch_gram(U, k, k, U, k, k, m, fdt, ctx->part, ctx->Gu, s);
    launch_gram(V, k, k, V, k, k, n, fdt, ctx->part, ctx->Gv, s);
    launch_dot(ctx->Gu, k, ctx->Gv, k, k, k, T_F64, ctx->part, &ctx->scal[11], s);
  }
  enmf_status rc = check_launch(ctx);
  if (rc) return rc;
  double h[4];
  CK(cudaMemcpyAsync(h, &ctx->scal[8], 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  rc = sync_status(ctx);
  if (rc) return rc;
  double e2 = dense_direct ? h[1] : h[0] - 2.0 * h[2] + h[3];
  out3[0] = 0.5 * e2;
  out3[1] = h[0] > 0 ? sqrt(e2 > 0 ? e2 : 0.0) / sqrt(h[0]) : 0.0;
  out3[2] = h[0];
  return ENMF_OK;
}

// ----------------------------------------------------------------- 5. KKT
extern "C" enmf_status enmf_kkt(enmf_ctx* ctx, const void* X, const void* U, const void* V,
                                enmf_kkt_report* out) {
  GUARD(ctx);
  if (!X || !U || !V || !out) return ENMF_EINVAL;
  {
    const void* xb = nullptr;
    const enmf_status brc = bind_x(ctx, X, &xb);
    if (brc) return brc;
    X = xb;
  }
  const enmf_problem& p = ctx->p;
  const int k = p.r, fdt = ctx->fdt, xdt = ctx->xdt;
  const int64_t m = p.m, n = p.n;
  cudaStream_t s = ctx->stream;
  launch_xv(X, xdt, m, n, p.ldx, V, k, k, ctx->M0, k, fdt, ctx->splitk, ctx->num_sms, s);
  launch_xtu(X, xdt, m, n, p.ldx, U, k, k, ctx->N0, k, fdt, ctx->splitk, ctx->num_sms, s);
  launch_gram(U, k, k, U, k, k, m, fdt, ctx->part, ctx->Gu, s);
  launch_gram(V, k, k, V, k, k, n, fdt, ctx->part, ctx->Gv, s);
  launch_kkt_rows(U, ctx->M0, ctx->Gv, m, k, fdt, ctx->part, &ctx->scal[16], s);
  launch_kkt_rows(V, ctx->N0, ctx->Gu, n, k, fdt, ctx->part, &ctx->scal[24], s);
  launch_kkt_final(&ctx->scal[16], &ctx->scal[24], &ctx->scal[32], s);
  enmf_status rc = check_launch(ctx);
  if (rc) return rc;
  double h[6];
  CK(cudaMemcpyAsync(h, &ctx->scal[32], 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
  rc = sync_status(ctx);
  if (rc) return rc;
  out->min_w = h[0];
  out->min_grad = h[1];
  out->delta = h[2];
  out->sigma = h[3];
  out->pg_norm = h[4];
  out->pg_rel = h[5];
  return ENMF_OK;
}

// ------------------------------------------------------------- one call
static bool is_device_ptr(const void* q) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

extern "C" enmf_status enmf_solve(enmf_ctx* ctx, const void* X, void* U, void* V, int32_t n_iter,
                                  const enmf_svd_opts* svd, const enmf_admm_opts* admm,
                                  const enmf_iter_opts* iter, double* out3) {
  GUARD(ctx);
  if (!X || !U || !V || n_iter < 0) return ENMF_EINVAL;
  const enmf_problem& p = ctx->p;
  if (ctx->xdt == T_CSR) {
    // the sparse form takes device arrays only (the descriptor is host memory)
    const enmf_csr* d = (const enmf_csr*)X;
    if (!is_device_ptr(U) || !is_device_ptr(V) || !d->row_ptr || !is_device_ptr(d->row_ptr) ||
        (p.nnz > 0 && (!is_device_ptr(d->col) || !is_device_ptr(d->val))))
      return ENMF_EINVAL;
    enmf_status rc = enmf_svd_init(ctx, X, U, V, nullptr, svd, nullptr);
    if (rc && rc != ENMF_ENOTCONV) return rc;
    rc = enmf_rotate(ctx, U, V, nullptr, admm, nullptr);
    if (rc && rc != ENMF_ENOTCONV) return rc;
    enmf_iter_opts io = {n_iter, 5, 1e-4, 3, nullptr, 1, 0, 10};
    if (iter) {
      io = *iter;
      io.n_iter = n_iter;
      io.reset = 1;
      io.sync_info = 0;
    }
    rc = enmf_iterate(ctx, X, U, V, &io, nullptr);
    if (rc) return rc;
    double o3[3];
    rc = enmf_residual(ctx, X, U, V, o3, 1);
    if (rc) return rc;
    if (out3) memcpy(out3, o3, sizeof(o3));
    return ENMF_OK;
  }
  const size_t xs = type_size(ctx->xdt), fs = type_size(ctx->fdt);
  const size_t xbytes = (size_t)((p.m - 1) * p.ldx + p.n) * xs;
  const size_t ub = (size_t)p.m * p.r * fs, vb = (size_t)p.n * p.r * fs;
  cudaStream_t s = ctx->stream;
  const void* dX = X;
  void* dU = U;
  void* dV = V;
  bool hostU = !is_device_ptr(U), hostV = !is_device_ptr(V);
  if (!is_device_ptr(X)) {
    if (!ctx->hX || ctx->hX_bytes < xbytes) {
      if (ctx->hX) cudaFree(ctx->hX);
      ctx->hX = nullptr;
      if (cudaMalloc(&ctx->hX, xbytes) != cudaSuccess) { cudaGetLastError(); return ENMF_ENOMEM; }
      ctx->hX_bytes = xbytes;
    }
    CK(cudaMemcpyAsync(ctx->hX, X, xbytes, cudaMemcpyHostToDevice, s));
    dX = ctx->hX;
  }
  if (hostU) {
    if (!ctx->hU && cudaMalloc(&ctx->hU, ub) != cudaSuccess) { cudaGetLastError(); return ENMF_ENOMEM; }
    dU = ctx->hU;
  }
  if (hostV) {
    if (!ctx->hV && cudaMalloc(&ctx->hV, vb) != cudaSuccess) { cudaGetLastError(); return ENMF_ENOMEM; }
    dV = ctx->hV;
  }
  enmf_status rc = ENMF_OK;
  if (ctx->tc) {
    rc = enmf_stage_x(ctx, dX);
    if (rc) return rc;
  }
  rc = enmf_svd_init(ctx, dX, dU, dV, nullptr, svd, nullptr);
  if (rc && rc != ENMF_ENOTCONV) return rc;
  rc = enmf_rotate(ctx, dU, dV, nullptr, admm, nullptr);
  if (rc && rc != ENMF_ENOTCONV) return rc;
  enmf_iter_opts io = {n_iter, 5, 1e-4, 3, nullptr, 1, 0, 10};
  if (iter) {
    io = *iter;
    io.n_iter = n_iter;
    io.reset = 1;
    io.sync_info = 0;
  }
  rc = enmf_iterate(ctx, dX, dU, dV, &io, nullptr);
  if (rc) return rc;
  double o3[3];
  rc = enmf_residual(ctx, dX, dU, dV, o3, 1);
  if (rc) return rc;
  if (hostU) CK(cudaMemcpyAsync(U, dU, ub, cudaMemcpyDeviceToHost, s));
  if (hostV) CK(cudaMemcpyAsync(V, dV, vb, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (out3) memcpy(out3, o3, sizeof(o3));
  return ENMF_OK;
}

// ------------------------------------- matrix completion (App. C, eNMC)
// Per-row masked Grams G (rows x KP x KP) and right-hand sides A (rows x KP)
// for the larger side, from the stream-ordered allocator for one call.
static enmf_status nmc_work(enmf_ctx* ctx, int gdt, void** G, void** A) {
  const enmf_problem& p = ctx->p;
  const int64_t rows = p.m > p.n ? p.m : p.n;
  const size_t kp = (size_t)nmc_rank_pad(p.r), fs = type_size(gdt);
  const size_t gb = al256((size_t)rows * kp * kp * fs), ab = al256((size_t)rows * kp * fs);
  void* w = nullptr;
  if (cudaMallocAsync(&w, gb + ab, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return ENMF_ENOMEM;
  }
  *G = w;
  *A = (char*)w + gb;
  return ENMF_OK;
}

// The rows of one side as compressed rows of the known entries: U's rows are
// X's rows, V's rows are the transpose's.
static void nmc_side(enmf_ctx* ctx, int which, const int64_t** rp, const int32_t** ix,
                     const void** val, int64_t* rows) {
  const CsrX& x = ctx->sx;
  *rp = which == 0 ? x.row_ptr : x.col_ptr;
  *ix = which == 0 ? x.col : x.row_t;
  *val = which == 0 ? x.val : x.val_t;
  *rows = which == 0 ? x.m : x.n;
}

extern "C" enmf_status enmf_nmc_objective(enmf_ctx* ctx, const void* X, const void* U,
                                          const void* V, double* out2) {
  GUARD(ctx);
  if (!X || !U || !V || !out2) return ENMF_EINVAL;
  if (ctx->xdt != T_CSR) return ENMF_ESTATE;
  {
    const void* xb = nullptr;
    const enmf_status brc = bind_x(ctx, X, &xb);
    if (brc) return brc;
  }
  cudaStream_t s = ctx->stream;
  launch_csr_normx2(ctx->sx, ctx->part, &ctx->scal[8], ctx->err, s);
  launch_nmc_objective(ctx->sx, U, V, ctx->p.r, ctx->fdt, 1.0, ctx->part, &ctx->scal[9], s);
  enmf_status rc = check_launch(ctx);
  if (rc) return rc;
  double h[2];
  CK(cudaMemcpyAsync(h, &ctx->scal[8], 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  rc = sync_status(ctx);
  if (rc) return rc;
  out2[0] = 0.5 * h[1];
  out2[1] = h[0] > 0 ? sqrt(h[1] / h[0]) : 0.0;
  return ENMF_OK;
}

extern "C" enmf_status enmf_nmc_start(enmf_ctx* ctx, const void* X, void* U, void* V,
                                      const enmf_nmc_start_opts* opts,
                                      enmf_nmc_start_info* info) {
  GUARD(ctx);
  if (!X || !U || !V) return ENMF_EINVAL;
  if (ctx->xdt != T_CSR) return ENMF_ESTATE;
  enmf_nmc_start_opts o = {50, 1e-3, 1e-10, 0};
  if (opts) {
    o = *opts;
    if (o.max_sweeps < 0 || !(o.lam >= 0) || !(o.tol >= 0) || o.svd_max_iters < 0)
      return ENMF_EINVAL;
  }
  // the balanced truncated SVD of the zero-filled X (the stored entries)
  enmf_svd_opts so = {10, 40, ctx->fdt == T_F64 ? 1e-12 : 1e-5, 0x5eedull};
  if (o.svd_max_iters > 0) so.max_iters = o.svd_max_iters;
  enmf_status rc = enmf_svd_init(ctx, X, U, V, nullptr, &so, nullptr);
  if (rc && rc != ENMF_ENOTCONV) return rc;
  void *G = nullptr, *A = nullptr;
  rc = nmc_work(ctx, T_F64, &G, &A);
  if (rc) return rc;
  cudaStream_t s = ctx->stream;
  const int k = ctx->p.r, fdt = ctx->fdt;
  bool notconv = false;   // a row's matrix was not positive definite (sticky)
  auto objective = [&](double* f) -> enmf_status {
    launch_nmc_objective(ctx->sx, U, V, k, fdt, 0.5, ctx->part, &ctx->scal[12], s);
    enmf_status e = check_launch(ctx);
    if (e) return e;
    CK(cudaMemcpyAsync(f, &ctx->scal[12], sizeof(double), cudaMemcpyDeviceToHost, s));
    e = sync_status(ctx);
    if (e == ENMF_ENOTCONV) {
      notconv = true;
      e = ENMF_OK;
    }
    return e;
  };
  double f_old = 0.0, f = 0.0;
  int sw = 0;
  rc = objective(&f_old);
  f = f_old;
  for (int it = 1; it <= o.max_sweeps && rc == ENMF_OK; ++it) {
    for (int which = 0; which < 2; ++which) {
      const int64_t* rp;
      const int32_t* ix;
      const void* val;
      int64_t rows;
      nmc_side(ctx, which, &rp, &ix, &val, &rows);
      void* F = which == 0 ? U : V;
      const void* Bf = which == 0 ? V : U;
      launch_nmc_gram(rp, ix, val, rows, Bf, k, fdt, T_F64, G, A, ctx->num_sms, s);
      launch_nmc_solve(G, A, rows, k, o.lam, F, fdt, ctx->err, ctx->num_sms, s);
    }
    sw = it;
    rc = objective(&f);
    if (rc) break;
    if (fabs(f_old - f) <= o.tol * fabs(f)) break;
    f_old = f;
  }
  cudaFreeAsync(G, s);
  ctx->state_valid = false;
  ctx->hals_known = false;
  if (rc == ENMF_OK) rc = sync_status(ctx);
  if (info) {
    info->sweeps = sw;
    info->f = f;
  }
  if (rc == ENMF_OK && notconv) rc = ENMF_ENOTCONV;
  return rc;
}

extern "C" enmf_status enmf_nmc_iterate(enmf_ctx* ctx, const void* X, void* U, void* V,
                                        const enmf_iter_opts* opts, enmf_iter_info* info) {
  GUARD(ctx);
  if (!X || !U || !V) return ENMF_EINVAL;
  if (ctx->xdt != T_CSR) return ENMF_ESTATE;
  enmf_iter_opts o = {0, 5, 1e-4, 3, nullptr, 0, 1, 10};
  if (opts) o = *opts;
  if (o.n_iter < 0 || o.pbcd_max_iter < 0 || !(o.eps >= 0) || o.n_shift < 1) return ENMF_EINVAL;
  {
    const void* xb = nullptr;
    const enmf_status brc = bind_x(ctx, X, &xb);
    if (brc) return brc;
  }
  void *G = nullptr, *A = nullptr;
  enmf_status rc = nmc_work(ctx, ctx->fdt, &G, &A);
  if (rc) return rc;
  const enmf_problem& p = ctx->p;
  const int k = p.r, fdt = ctx->fdt;
  cudaStream_t s = ctx->stream;
  if (o.reset || !ctx->state_valid) {
    // the Eq. 8 / 9 steps from the negative maxima of the current U, V
    launch_state_init(U, V, p.m, p.n, k, fdt, o.n_shift, ctx->st, ctx->part, s);
    ctx->state_valid = true;
    ctx->hals_known = false;
    ctx->nmc_rounds = 0;
  }
  for (int it = 0; it < o.n_iter; ++it) {
    for (int which = 0; which < 2; ++which) {
      const int64_t* rp;
      const int32_t* ix;
      const void* val;
      int64_t rows;
      nmc_side(ctx, which, &rp, &ix, &val, &rows);
      void* F = which == 0 ? U : V;
      const void* Bf = which == 0 ? V : U;
      launch_nmc_gram(rp, ix, val, rows, Bf, k, fdt, fdt, G, A, ctx->num_sms, s);
      NmcArgs a;
      memset(&a, 0, sizeof(a));
      a.F = F;
      a.gbuf = ctx->Zb;
      a.G = G;
      a.A = A;
      a.mask = ctx->mask;
      a.part = ctx->part;
      a.bar = &ctx->st->bar;
      a.err = ctx->err;
      a.st = ctx->st;
      a.rows = rows;
      a.k = k;
      a.fdt = fdt;
      a.which = which;
      a.round = ctx->nmc_rounds;
      a.pbcd_max_iter = o.pbcd_max_iter;
      a.eps = o.eps;
      launch_nmc_pbcd(a, nmc_pbcd_grid(fdt, k, ctx->num_sms, rows), s);
    }
    launch_nmc_objective(ctx->sx, U, V, k, fdt, 0.5, ctx->part,
                         o.trace ? o.trace + it : &ctx->st->f_last, s);
    ++ctx->nmc_rounds;
    rc = check_launch(ctx);
    if (rc) break;
  }
  cudaFreeAsync(G, s);
  if (rc) return rc;
  if (o.sync_info || info) {
    rc = sync_status(ctx);
    if (rc) return rc;
    if (info) {
      memset(info, 0, sizeof(*info));
      info->iters = ctx->nmc_rounds;
      info->asc_iters = ctx->nmc_rounds;
      DevState hst;
      CK(cudaMemcpy(&hst, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost));
      info->s_u = hst.s_u;
      info->s_v = hst.s_v;
    }
  }
  return ENMF_OK;
}
