// Batching: many problems of the tensor-core form iterated together, every
// phase of every alternation one grouped launch over all members:
//   [X_lo passes]  X V sweep  ->  U-half  ->  [X_lo passes]  X^T U sweep  ->  V-half
// The sweeps are the stream-K tensor-core kernel over the concatenated work of
// all members (tc_sweep.cu); the half steps are the grouped cooperative
// kernel (hstep.cu), each member on its own group of blocks with one grid
// barrier for all.  A step of several alternations is captured once as a
// CUDA graph and replayed while the membership is unchanged.  The grid of the
// grouped sweeps is picked by timing candidates on the live membership
// (enmf_batch_tune).
#include <string.h>

#include <new>
#include <vector>

#include "ctx.h"

struct enmf_batch {
  cudaStream_t stream;
  enmf_iter_opts o;
  int max_members;
  int num_sms;
  int rp;                 // padded rank of every member (0 until the first add)
  struct Member {
    enmf_ctx* ctx;
    const void* X;
    void* U;
    void* V;
    bool used;
  };
  std::vector<Member> mem;
  int n_active;
  bool dirty;             // membership changed since the descriptors were built
  long long alt;          // alternations run by the batch
  // device memory: descriptors, block tables, barrier, stream-K slots
  void* dmem;
  SweepProb* d_sw[4];     // X V main, X V lo, X^T U main, X^T U lo
  HalfArgs* d_half[2];    // U-half, V-half
  int* d_bbeg[2];
  GridBarrier* d_bar;
  int* d_err;             // status word of the grouped sweeps (bounded waits)
  float* part;
  int* counters;
  int64_t counters_cap;
  // host mirrors of the descriptors
  std::vector<SweepProb> h_sw[4];
  std::vector<HalfArgs> h_half[2];
  std::vector<int> h_bbeg[2];
  int np[4];
  int64_t W[4];
  int half_grid[2];
  int sweep_grid;         // 0: one CTA per SM (or fewer); else the tuned grid
  int sweep_stages;       // X ring depth of the sweeps: 0 = as deep as fits; else tuned
  // the captured step
  cudaStream_t cap;
  cudaGraphExec_t graph;
  int graph_nalt, graph_phase, graph_kernels;
  bool no_graph;
  // enmf_batch_states: the members' DevState pointers and a gathered copy
  // of their states (device), read back in one copy into pinned host memory
  DevState** d_stp;
  DevState* d_gather;
  DevState* h_gather;
  int gather_cap;
};

namespace {

void batch_free(enmf_batch* b) {
  if (b->d_stp) cudaFree(b->d_stp);
  if (b->d_gather) cudaFree(b->d_gather);
  if (b->h_gather) cudaFreeHost(b->h_gather);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->counters) cudaFree(b->counters);
  if (b->dmem) cudaFree(b->dmem);
  delete b;
}

// Blocks of each member's half step: one per 32 rows (at most NPART), scaled
// down when the total exceeds the co-resident capacity of the grouped kernel.
void split_blocks(const std::vector<int64_t>& rows, int cap, std::vector<int>& bbeg) {
  const int np = (int)rows.size();
  std::vector<int> nb(np);
  long long total = 0;
  for (int p = 0; p < np; ++p) {
    int64_t need = (rows[p] + 31) / 32;
    if (need > NPART) need = NPART;
    nb[p] = (int)(need < 1 ? 1 : need);
    total += nb[p];
  }
  while (total > cap) {   // take one block from the member with the most
    int pm = 0;
    for (int p = 1; p < np; ++p)
      if (nb[p] > nb[pm]) pm = p;
    if (nb[pm] <= 1) break;
    --nb[pm];
    --total;
  }
  bbeg.assign(np + 1, 0);
  for (int p = 0; p < np; ++p) bbeg[p + 1] = bbeg[p] + nb[p];
}

enmf_status rebuild(enmf_batch* b) {
  for (int q = 0; q < 4; ++q) {
    b->h_sw[q].clear();
    b->W[q] = 0;
  }
  b->h_half[0].clear();
  b->h_half[1].clear();
  std::vector<int64_t> rows_u, rows_v;
  int64_t tiles[4] = {0, 0, 0, 0};
  for (auto& mb : b->mem) {
    if (!mb.used) continue;
    enmf_ctx* ctx = mb.ctx;
    const enmf_problem& p = ctx->p;
    for (int q = 0; q < 4; ++q) {
      const int mode = q < 2 ? 0 : 1;
      const bool lo = q & 1;
      if (lo && !ctx->xl) continue;
      SweepProb d;
      memset(&d, 0, sizeof(d));
      memcpy(d.mapX, ctx->maps[lo ? MAP_XL : MAP_XH], sizeof(d.mapX));
      memcpy(d.mapBh, ctx->maps[mode == 0 ? MAP_VH : MAP_UH], sizeof(d.mapBh));
      memcpy(d.mapBl, ctx->maps[mode == 0 ? MAP_VL : MAP_UL], sizeof(d.mapBl));
      int64_t units, t;
      tc_prob_sizes(mode, &d, mode == 0 ? p.m : p.n, mode == 0 ? p.n : p.m, p.r, b->W[q],
                    tiles[q], &units, &t);
      float* main_out = (float*)(mode == 0 ? ctx->M0 : ctx->N0);
      float* lo_out = mode == 0 ? ctx->cv : ctx->cu;
      d.out = lo ? lo_out : main_out;
      d.corr = (!lo && ctx->xl) ? lo_out : nullptr;
      d.f16 = ctx->tf16;
      d.l2hint = lo ? 2 : 0;   // X_lo is read once per correction period
      b->h_sw[q].push_back(d);
      b->W[q] += units;
      tiles[q] += t;
    }
    HalfArgs hu = ctx_half_args(ctx, 0, mb.U, ctx->M0, ctx->Gv, p.m, b->o, false, ctx->Gu,
                                nullptr, nullptr, 0);
    HalfArgs hv = ctx_half_args(ctx, 1, mb.V, ctx->N0, ctx->Gu, p.n, b->o, true, ctx->Gv,
                                ctx->Gu, nullptr, 0);
    hu.bar = b->d_bar;
    hv.bar = b->d_bar;
    b->h_half[0].push_back(hu);
    b->h_half[1].push_back(hv);
    rows_u.push_back(p.m);
    rows_v.push_back(p.n);
  }
  for (int q = 0; q < 4; ++q) b->np[q] = (int)b->h_sw[q].size();
  const int cap = half_group_capacity(b->rp, b->num_sms);
  split_blocks(rows_u, cap, b->h_bbeg[0]);
  split_blocks(rows_v, cap, b->h_bbeg[1]);
  b->half_grid[0] = b->h_bbeg[0].back();
  b->half_grid[1] = b->h_bbeg[1].back();
  // per-tile arrival counters: the largest launch's tile count
  int64_t need = 1;
  for (int q = 0; q < 4; ++q) need = tiles[q] > need ? tiles[q] : need;
  if (need > b->counters_cap) {
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return ENMF_ECUDA;
    if (b->counters) cudaFree(b->counters);
    b->counters = nullptr;
    b->counters_cap = 0;
    if (cudaMalloc(&b->counters, (size_t)need * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return ENMF_ENOMEM;
    }
    b->counters_cap = need;
    if (cudaMemsetAsync(b->counters, 0, (size_t)need * sizeof(int), b->stream) != cudaSuccess)
      return ENMF_ECUDA;
  }
  for (int q = 0; q < 4; ++q)
    if (b->np[q] &&
        cudaMemcpyAsync(b->d_sw[q], b->h_sw[q].data(), b->np[q] * sizeof(SweepProb),
                        cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
      return ENMF_ECUDA;
  for (int h = 0; h < 2; ++h) {
    const int n = (int)b->h_half[h].size();
    if (n && (cudaMemcpyAsync(b->d_half[h], b->h_half[h].data(), n * sizeof(HalfArgs),
                              cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
              cudaMemcpyAsync(b->d_bbeg[h], b->h_bbeg[h].data(), (n + 1) * sizeof(int),
                              cudaMemcpyHostToDevice, b->stream) != cudaSuccess))
      return ENMF_ECUDA;
  }
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->dirty = false;
  return ENMF_OK;
}

void sweep(enmf_batch* b, int q, int grid, int stages) {
  if (!b->np[q]) return;
  launch_tc_group(q < 2 ? 0 : 1, b->rp, b->d_sw[q], b->np[q], b->W[q], b->part, b->counters,
                  grid > 0 ? grid : b->num_sms, b->d_err, b->stream, 1, 0, stages);
}

// One alternation of every member (refreshing the X_lo terms when corr).
void alternation(enmf_batch* b, bool corr) {
  const int np = (int)b->h_half[0].size();
  if (corr) sweep(b, 1, b->sweep_grid, b->sweep_stages);
  sweep(b, 0, b->sweep_grid, b->sweep_stages);
  launch_half_group(b->d_half[0], b->d_bbeg[0], np, b->half_grid[0], b->rp, b->stream);
  if (corr) sweep(b, 3, b->sweep_grid, b->sweep_stages);
  sweep(b, 2, b->sweep_grid, b->sweep_stages);
  launch_half_group(b->d_half[1], b->d_bbeg[1], np, b->half_grid[1], b->rp, b->stream);
}

void run_step(enmf_batch* b, int n_alt) {
  for (int j = 0; j < n_alt; ++j) alternation(b, (b->alt + j) % b->o.correct_every == 0);
}

}  // namespace

extern "C" enmf_status enmf_batch_create(const enmf_iter_opts* opts, int32_t max_members,
                                         void* stream, enmf_batch** out) {
  if (!out || max_members < 1 || max_members > 4096) return ENMF_EINVAL;
  enmf_iter_opts o = {0, 5, 1e-4, 3, nullptr, 0, 0, 10};
  if (opts) o = *opts;
  if (o.pbcd_max_iter < 0 || !(o.eps >= 0) || o.n_shift < 1) return ENMF_EINVAL;
  if (o.correct_every < 1) o.correct_every = 10;
  enmf_batch* b = new (std::nothrow) enmf_batch();
  if (!b) return ENMF_ENOMEM;
  b->stream = (cudaStream_t)stream;
  b->o = o;
  b->max_members = max_members;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return ENMF_ECUDA;
  }
  b->mem.resize(max_members);
  const size_t mm = (size_t)max_members;
  const size_t sw = mm * sizeof(SweepProb), ha = mm * sizeof(HalfArgs), bb = (mm + 1) * sizeof(int);
  const size_t part = (size_t)b->num_sms * 2 * 128 * 64 * sizeof(float);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t total = 4 * al(sw) + 2 * al(ha) + 2 * al(bb) + al(sizeof(GridBarrier)) +
                       al(sizeof(int)) + al(part);
  if (cudaMalloc(&b->dmem, total) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return ENMF_ENOMEM;
  }
  cudaMemsetAsync(b->dmem, 0, total, b->stream);
  char* q = (char*)b->dmem;
  for (int i = 0; i < 4; ++i, q += al(sw)) b->d_sw[i] = (SweepProb*)q;
  for (int i = 0; i < 2; ++i, q += al(ha)) b->d_half[i] = (HalfArgs*)q;
  for (int i = 0; i < 2; ++i, q += al(bb)) b->d_bbeg[i] = (int*)q;
  b->d_bar = (GridBarrier*)q;
  q += al(sizeof(GridBarrier));
  b->d_err = (int*)q;
  q += al(sizeof(int));
  b->part = (float*)q;
  *out = b;
  return ENMF_OK;
}

extern "C" void enmf_batch_destroy(enmf_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
}

extern "C" enmf_status enmf_batch_add(enmf_batch* b, enmf_ctx* ctx, const void* X, void* U, void* V,
                                      int32_t* slot) {
  if (!b || !ctx || !X || !U || !V || !slot) return ENMF_EINVAL;
  if (ctx->poison) return ctx->poison;
  if (!ctx->tc || ctx->staged_src != X) return ENMF_ESTATE;
  if (ctx->xq) return ENMF_EINVAL;   // the FP8 form iterates alone
  const int rp = tc_rank_pad(ctx->p.r);
  if (b->rp && rp != b->rp) return ENMF_EINVAL;
  if (b->n_active >= half_group_capacity(rp, b->num_sms)) return ENMF_EBUSY;
  int s = -1;
  for (int i = 0; i < b->max_members; ++i)
    if (!b->mem[i].used) {
      s = i;
      break;
    }
  if (s < 0) return ENMF_EBUSY;
  for (auto& mb : b->mem)
    if (mb.used && mb.ctx == ctx) return ENMF_EINVAL;
  // the member's own ascent stage, alone on its stream, exactly as
  // enmf_iterate runs a fresh one (n_shift alternations, the X_lo term
  // refreshed in each); then its descent joins the batch.  The batch stream
  // waits for it (and for the caller's earlier work on that stream).
  {
    enmf_iter_opts io = b->o;
    io.n_iter = b->o.n_shift;
    io.trace = nullptr;
    io.reset = 1;
    io.sync_info = 0;
    const enmf_status rc0 = enmf_iterate(ctx, X, U, V, &io, nullptr);
    if (rc0) return rc0;
  }
  ctx_iter_prologue(ctx, X, U, V, b->o.n_shift, false);
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return ENMF_ECUDA;
  }
  cudaEventRecord(ev, ctx->stream);
  cudaStreamWaitEvent(b->stream, ev, 0);
  cudaEventDestroy(ev);
  enmf_status rc = ctx_check_launch(ctx);
  if (rc) return rc;
  b->rp = rp;
  b->mem[s] = {ctx, X, U, V, true};
  ++b->n_active;
  b->dirty = true;
  *slot = s;
  return ENMF_OK;
}

extern "C" enmf_status enmf_batch_remove(enmf_batch* b, int32_t slot) {
  if (!b || slot < 0 || slot >= b->max_members || !b->mem[slot].used) return ENMF_EINVAL;
  // the member's stream waits for the batch's work on it
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return ENMF_ECUDA;
  }
  cudaEventRecord(ev, b->stream);
  cudaStreamWaitEvent(b->mem[slot].ctx->stream, ev, 0);
  cudaEventDestroy(ev);
  b->mem[slot].used = false;
  --b->n_active;
  if (b->n_active == 0) b->rp = 0;
  b->dirty = true;
  return ENMF_OK;
}

extern "C" int32_t enmf_batch_size(const enmf_batch* b) { return b ? b->n_active : 0; }

extern "C" enmf_status enmf_batch_step(enmf_batch* b, int32_t n_alt) {
  if (!b || n_alt < 0 || n_alt % b->o.correct_every != 0) return ENMF_EINVAL;
  if (n_alt == 0 || b->n_active == 0) return ENMF_OK;
  if (b->dirty) {
    enmf_status rc = rebuild(b);
    if (rc) return rc;
  }
  const int phase = (int)(b->alt % b->o.correct_every);
  bool done = false;
  if (!b->no_graph && n_alt >= 2) {
    if (!b->graph || b->graph_nalt != n_alt || b->graph_phase != phase) {
      if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
      }
      bool ok = b->cap || cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
      cudaGraph_t g = nullptr;
      const long long l0 = enmf_launch_count();
      if (ok) ok = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        cudaStream_t user = b->stream;
        b->stream = b->cap;
        run_step(b, n_alt);
        b->stream = user;
        ok = cudaStreamEndCapture(b->cap, &g) == cudaSuccess && g;
      }
      const int kernels = (int)(enmf_launch_count() - l0);
      note_launch(-kernels);   // captured, not launched
      cudaGraphExec_t exec = nullptr;
      if (ok) ok = cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
      if (g) cudaGraphDestroy(g);
      if (ok) {
        b->graph = exec;
        b->graph_nalt = n_alt;
        b->graph_phase = phase;
        b->graph_kernels = kernels;
      } else {
        cudaGetLastError();
        b->no_graph = true;
      }
    }
    if (b->graph) {
      if (cudaGraphLaunch(b->graph, b->stream) == cudaSuccess) {
        note_launch(b->graph_kernels);
        done = true;
      } else {
        cudaGetLastError();
        b->no_graph = true;
      }
    }
  }
  if (!done) run_step(b, n_alt);
  b->alt += n_alt;
  return cudaGetLastError() == cudaSuccess ? ENMF_OK : ENMF_ECUDA;
}

extern "C" enmf_status enmf_batch_member(enmf_batch* b, int32_t slot, enmf_iter_info* info,
                                         double* f) {
  if (!b || slot < 0 || slot >= b->max_members || !b->mem[slot].used) return ENMF_EINVAL;
  enmf_ctx* ctx = b->mem[slot].ctx;
  DevState hst;
  int berr = 0;
  if (cudaMemcpyAsync(&hst, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(&berr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess) {
    cudaGetLastError();
    return ENMF_ECUDA;
  }
  if (berr & ERR_TIMEOUT) return ENMF_ETIMEOUT;
  enmf_status rc = ctx_sync_status(ctx);
  if (info) {
    info->iters = hst.k;
    info->asc_iters = hst.asc_iters;
    info->hals_iters = hst.hals_iters;
    info->stage = hst.stage;
    info->s_u = hst.s_u;
    info->s_v = hst.s_v;
  }
  if (f) *f = hst.f_last;
  return rc;
}

namespace {
// out[i] = *stp[i] for the members listed in stp (one thread block per member).
__global__ void gather_states_kernel(DevState* const* __restrict__ stp, int n, DevState* out) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const int words = (int)(sizeof(DevState) / sizeof(int));
  const int* src = reinterpret_cast<const int*>(stp[i]);
  int* dst = reinterpret_cast<int*>(out + i);
  for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
}
}  // namespace

extern "C" enmf_status enmf_batch_states(enmf_batch* b, int32_t* slots, enmf_iter_info* infos,
                                         double* f, int32_t cap, int32_t* count) {
  if (!b || !count || cap < 0 || (cap > 0 && (!slots || !infos || !f))) return ENMF_EINVAL;
  std::vector<int> sl;
  std::vector<DevState*> stp;
  for (int q = 0; q < b->max_members; ++q)
    if (b->mem[q].used) {
      sl.push_back(q);
      stp.push_back(b->mem[q].ctx->st);
    }
  const int n = (int)sl.size();
  *count = n;
  if (n == 0) return ENMF_OK;
  if (cap < n) return ENMF_EINVAL;
  if (b->gather_cap < n) {
    if (b->d_stp) cudaFree(b->d_stp);
    if (b->d_gather) cudaFree(b->d_gather);
    if (b->h_gather) cudaFreeHost(b->h_gather);
    b->d_stp = nullptr;
    b->d_gather = nullptr;
    b->h_gather = nullptr;
    b->gather_cap = 0;
    const int c = b->max_members;
    if (cudaMalloc(&b->d_stp, sizeof(DevState*) * c) != cudaSuccess ||
        cudaMalloc(&b->d_gather, sizeof(DevState) * c) != cudaSuccess ||
        cudaMallocHost(&b->h_gather, sizeof(DevState) * c) != cudaSuccess) {
      cudaGetLastError();
      return ENMF_ENOMEM;
    }
    b->gather_cap = c;
  }
  int berr = 0;
  if (cudaMemcpyAsync(b->d_stp, stp.data(), sizeof(DevState*) * n, cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess) {
    cudaGetLastError();
    return ENMF_ECUDA;
  }
  note_launch(1);
  gather_states_kernel<<<n, 32, 0, b->stream>>>(b->d_stp, n, b->d_gather);
  if (cudaMemcpyAsync(b->h_gather, b->d_gather, sizeof(DevState) * n, cudaMemcpyDeviceToHost,
                      b->stream) != cudaSuccess ||
      cudaMemcpyAsync(&berr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess) {
    cudaGetLastError();
    return ENMF_ECUDA;
  }
  if (berr & ERR_TIMEOUT) return ENMF_ETIMEOUT;
  for (int i = 0; i < n; ++i) {
    const DevState& h = b->h_gather[i];
    slots[i] = sl[i];
    infos[i].iters = h.k;
    infos[i].asc_iters = h.asc_iters;
    infos[i].hals_iters = h.hals_iters;
    infos[i].stage = h.stage;
    infos[i].s_u = h.s_u;
    infos[i].s_v = h.s_v;
    f[i] = h.f_last;
  }
  return ENMF_OK;
}

extern "C" enmf_status enmf_batch_tune(enmf_batch* b, int32_t* grid_out, float* ms_out) {
  if (!b) return ENMF_EINVAL;
  if (b->n_active == 0) return ENMF_OK;
  if (b->dirty) {
    enmf_status rc = rebuild(b);
    if (rc) return rc;
  }
  // candidates: the stream-K grid of the grouped sweeps x the depth of their
  // shared-memory ring of X stages (2, 3, or as deep as fits)
  const int cands[4] = {b->num_sms / 4, b->num_sms / 2, (3 * b->num_sms) / 4, b->num_sms};
  const int st_cands[3] = {2, 3, 0};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return ENMF_ECUDA;
  }
  int best = 0, best_st = 0;
  float best_ms = 1e30f;
  for (int c = 0; c < 4; ++c)
    for (int si = 0; si < 3; ++si) {
      const int g = cands[c] < 1 ? 1 : cands[c];
      const int st = st_cands[si];
      // X V and X^T U sweeps alone: they read the current factors and write
      // the members' sweep outputs, which the next alternation overwrites
      sweep(b, 0, g, st);
      sweep(b, 2, g, st);
      cudaEventRecord(e0, b->stream);
      for (int rep = 0; rep < 3; ++rep) {
        sweep(b, 0, g, st);
        sweep(b, 2, g, st);
      }
      cudaEventRecord(e1, b->stream);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = g;
        best_st = st;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best > 0 && (best != b->sweep_grid || best_st != b->sweep_stages)) {
    b->sweep_grid = best;
    b->sweep_stages = best_st;
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
  }
  if (grid_out) *grid_out = b->sweep_grid;
  if (ms_out) *ms_out = best_ms / 3.f;
  return cudaGetLastError() == cudaSuccess ? ENMF_OK : ENMF_ECUDA;
}
