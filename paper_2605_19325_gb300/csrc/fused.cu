// One HALS alternation's U-half fused with both products of the core kernel
// (App. I) in a single pass over X: for every row panel P of X (128 rows),
//   A_P   = X_P V (+ X_lo,P V, the precision form's correction term),
//   U_P  <- HALS(U_P, A_P, V^T V)      (Sec. 4.3; rows are independent, Sec. 4.2),
//   X^T U += X_P^T U_P                  (with the NEW rows of U -- Gauss-Seidel),
// plus the Gram U^T U of the new factor.  The V-half then needs only the
// X^T U partials and U^T U (hstep.cu).  X is read from HBM once per
// alternation instead of twice.
//
// Thread-block cluster of C CTAs per row panel.  CTA j of a cluster owns the
// column slice J_j = [j S, j S + S) of X (S a multiple of 128):
//   * its slice of V (as the BF16 / FP16 pair V^T hi, lo) stays in shared
//     memory for the whole launch, so X V of a panel is C partial products;
//   * the partials of one panel meet in distributed shared memory: CTA j sums
//     the rows [j R, j R + R) (R = 128 / C) of all C partials in CTA order and
//     runs the HALS column sweep on those rows;
//   * every CTA pushes its new rows of U (as the 16-bit pair, in the swizzled
//     K-major layout of a tcgen05 operand) into every CTA's panel buffer;
//   * each CTA accumulates X_P^T U_P for its slice in tensor memory, all
//     panels of the cluster long (S / 128 accumulators of 128 x RP).
// Panels are dealt to the clusters round robin.  At the end each CTA writes
// its slice of the cluster's X^T U partial; the V-half sums the clusters'
// partials in cluster order.
//
// Pipeline: warp 0 issues TMA loads (the V slice once, then 32 KB X stages),
// warp 1 issues the MMAs, warps 2-5 run the epilogue (tensor memory ->
// shared memory, the cluster exchange, HALS, the push of U).  The MMA order is
// X V of panel p + LAG before X^T U of panel p, so the exchange and HALS of
// panel p overlap the X V stream of the next panels; the X^T U stages re-read
// X_P, which is still in L2.  Every wait is bounded; after a timeout every
// role stops at its next wait and the CTA leaves through the final cluster
// barrier once its own copies and MMAs have drained.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdlib.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace enmf {
namespace fz {

using namespace tc;

constexpr int TILE = 128;                   // panel rows; slice columns per X^T U accumulator
constexpr int KB = 128;                     // X columns per ring stage (two 64-column boxes)
constexpr uint32_t STAGE = TILE * KB * 2;   // 32 KB
constexpr int THREADS = 256;              // + warps 6-7: global writes of the new U rows
constexpr int STAMP_PANELS = 32;          // diagnostic stamps kept per CTA (shared memory)
constexpr int LAG = 2;                      // panels of X V issued ahead of X^T U
constexpr int NACC = LAG + 1;               // X V accumulators
constexpr int MAX_STAGES = 6;

struct Smem {
  size_t vres, ring, ubuf, xstg, gs, urow, total;
};

// Dynamic shared memory layout (offsets from a 1024-byte aligned base).
__host__ __device__ inline Smem smem_plan(int rp, int S, int C, int nst) {
  Smem s;
  size_t o = 0;
  s.vres = o;  o += 2 * (size_t)S * rp * 2;          // V^T slice, hi then lo
  s.ring = o;  o += (size_t)nst * STAGE;
  s.ubuf = o;  o += 2 * (size_t)TILE * rp * 2;       // U panel pair, hi then lo
  s.xstg = o;  o += (size_t)TILE * (rp + 4) * 4;     // X V partial of the panel
  s.gs = o;    o += (size_t)rp * rp * 4 + (size_t)rp * 4;   // V^T V (FP32) and 1 / G_jj
  s.urow = o;  o += 2 * (size_t)(TILE / C) * rp * 4;  // this CTA's new rows of U, by panel parity
  s.total = o + 1024;                                 // alignment slack
  return s;
}

// Bounded wait of the fused kernel: false after WAIT_BUDGET cycles, or as soon
// as the launch has recorded a timeout elsewhere (so one expired wait stops
// every CTA quickly).  The status word is polled only once a wait has lasted
// 2^20 cycles: thousands of waiting threads must not spin on one global word.
__device__ __forceinline__ bool fwait(uint64_t* bar, uint32_t parity, int* err, bool cluster_scope) {
  if (cluster_scope ? mbar_try_cluster(bar, parity) : mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  long long next = 1LL << 20;
  while (true) {
    if (cluster_scope ? mbar_try_cluster(bar, parity) : mbar_try(bar, parity)) return true;
    const long long dt = clock64() - t0;
    if (dt > next) {
      if (*(volatile int*)err & ERR_TIMEOUT) return false;
      next = dt + (1LL << 20);
    }
    if (dt > WAIT_BUDGET) {
      atomicOr(err, ERR_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ long long gtimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Diagnostic stamp (event ev of local panel pi) into shared memory when the
// launch records them (written out at the end: a global store here would
// lengthen the cluster-scope releases that follow it).
__device__ __forceinline__ void stamp(long long* sst, bool on, int pi, int ev) {
  if (on && pi <= STAMP_PANELS) sst[pi * 8 + ev] = gtimer();
}

__device__ __forceinline__ uint16_t to16b(float v, int f16) {
  if (f16) return __half_as_ushort(__float2half_rn(v));
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
__device__ __forceinline__ float from16b(uint16_t b, int f16) {
  if (f16) return __half2float(__ushort_as_half(b));
  return __bfloat162float(__ushort_as_bfloat16(b));
}

template <int RP>
__global__ void __launch_bounds__(THREADS, 1) fused_hals_kernel(const FusedDesc* __restrict__ fd,
                                                                int nst) {
  constexpr uint32_t IDESC_XV_BF = idesc_f16kind(TILE, RP, 0, 0);
  constexpr uint32_t IDESC_XV_H = idesc_f16kind(TILE, RP, 0, 1);
  constexpr uint32_t IDESC_XT_BF = idesc_f16kind(TILE, RP, 1, 0);
  constexpr uint32_t IDESC_XT_H = idesc_f16kind(TILE, RP, 1, 1);
  constexpr int XLD = RP + 4;          // xstg row stride (floats)
  constexpr int NV = RP / 32;          // float4 groups per lane (lane owns 4 NV columns)
  constexpr uint32_t ATOM = RP * 128;  // one 64-wide K atom of an RP-row operand

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[MAX_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[MAX_STAGES];
  __shared__ __align__(8) uint64_t vfull_bar;
  __shared__ __align__(8) uint64_t accf_bar[NACC];
  __shared__ __align__(8) uint64_t acce_bar[NACC];
  __shared__ __align__(8) uint64_t staged_bar[2];    // C arrivals: every CTA staged its partial
  __shared__ __align__(8) uint64_t consumed_bar[2];  // C arrivals: every CTA read my partial
  __shared__ __align__(8) uint64_t uready_bar[2];    // C arrivals: every CTA pushed its U rows
  __shared__ __align__(8) uint64_t ufree_bar[2];     // C arrivals: every CTA's X^T U MMAs done
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ __align__(8) uint64_t wready_bar[2];    // epilogue -> writers: rows of U ready
  __shared__ __align__(8) uint64_t wdone_bar[2];     // writers -> epilogue: rows written out
  __shared__ long long sst[(STAMP_PANELS + 1) * 8];
  __shared__ uint32_t tmem_slot;
  __shared__ int aborted;
  __shared__ int last_cta;

  const FusedDesc& d = *fd;
  const int C = d.C, S = d.S, T = d.T, Q = d.Q, r = d.r;
  const int Rc = TILE / C;
  const int64_t m = d.m, n = d.n;
  const uint32_t j = cluster_rank();
  const int q = (int)(blockIdx.x / (unsigned)C);
  const int npan = q < d.npanels ? (d.npanels - q + Q - 1) / Q : 0;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  const Smem L = smem_plan(RP, S, C, nst);
  uint8_t* const vres = smem + L.vres;
  uint8_t* const ring = smem + L.ring;
  uint8_t* const ubuf = smem + L.ubuf;
  float* const xstg = reinterpret_cast<float*>(smem + L.xstg);
  float* const Gs = reinterpret_cast<float*>(smem + L.gs);
  float* const ginv = Gs + RP * RP;
  float* const urow = reinterpret_cast<float*>(smem + L.urow);
  const CUtensorMap* mapX = reinterpret_cast<const CUtensorMap*>(d.mapX);
  const CUtensorMap* mapVh = reinterpret_cast<const CUtensorMap*>(d.mapVh);
  const CUtensorMap* mapVl = reinterpret_cast<const CUtensorMap*>(d.mapVl);

  if (threadIdx.x == 0) {
    prefetch_map(mapX);
    prefetch_map(mapVh);
    prefetch_map(mapVl);
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&vfull_bar, 1);
    for (int b = 0; b < NACC; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&staged_bar[b], C);
      mbar_init(&consumed_bar[b], C);
      mbar_init(&uready_bar[b], C);
      mbar_init(&ufree_bar[b], C);
      mbar_init(&wready_bar[b], 1);
      mbar_init(&wdone_bar[b], 1);
    }
    mbar_init(&drain_bar, 1);
    aborted = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int e = threadIdx.x; e < (STAMP_PANELS + 1) * 8; e += THREADS) sst[e] = 0;
  // The U panel buffer's rows r..RP-1 are never pushed: zero the whole buffer
  // once (before any peer can write into it: the cluster barrier below).
  for (int e = threadIdx.x; e < (int)(2 * TILE * RP * 2 / 16); e += THREADS)
    reinterpret_cast<uint4*>(ubuf)[e] = make_uint4(0u, 0u, 0u, 0u);
  // V^T V (FP64, r x r) as FP32, zero padded, and 1 / G_jj (0 where G_jj <= 0)
  for (int e = threadIdx.x; e < RP * RP; e += THREADS) {
    const int a = e / RP, b = e % RP;
    Gs[e] = (a < r && b < r) ? (float)d.Gv[a * r + b] : 0.f;
  }
  if (warp == 1) {
    const uint32_t need = (uint32_t)((NACC + T) * RP);
    const uint32_t cols = need <= 32 ? 32 : need <= 64 ? 64 : need <= 128 ? 128 : need <= 256 ? 256 : 512;
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(&tmem_slot)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  for (int jj = threadIdx.x; jj < RP; jj += THREADS) {
    const float g = Gs[jj * RP + jj];
    ginv[jj] = g > 0.f ? 1.f / g : 0.f;
  }
  // every CTA's barriers are initialised before any peer arrives on them
  cluster_sync_all();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t tmem_cols = (uint32_t)((NACC + T) * RP);
  const bool stamping = d.stamps != nullptr;
  if (threadIdx.x == 0) stamp(sst, stamping, STAMP_PANELS, 0);
  const uint16_t cmask = (uint16_t)((1u << C) - 1u);
  int* const err = d.err;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------- producer
      const int64_t col0 = (int64_t)j * S;
      mbar_expect_tx(&vfull_bar, 2u * (uint32_t)S * RP * 2u);
      for (int a = 0; a < S / 64; ++a) {
        tma_load(vres + (size_t)a * ATOM, mapVh, &vfull_bar, (int)(col0 + 64 * a), 0);
        tma_load(vres + (size_t)S * RP * 2 + (size_t)a * ATOM, mapVl, &vfull_bar,
                 (int)(col0 + 64 * a), 0);
      }
      int64_t i = 0;
      bool ok = true;
      for (int s = 0; ok && s < npan + LAG; ++s) {
        for (int part = 0; ok && part < 2; ++part) {
          // part 0: X V stages of panel s; part 1: X^T U stages of panel s - LAG
          const int pi = part == 0 ? s : s - LAG;
          if (pi < 0 || pi >= npan) continue;
          const int row0 = (q + pi * Q) * TILE;
          for (int t = 0; t < T; ++t, ++i) {
            const int slot = (int)(i % nst);
            const uint32_t ph = (uint32_t)(i / nst) & 1u;
            if (*(volatile int*)&aborted || !fwait(&empty_bar[slot], ph ^ 1u, err, false)) {
              aborted = 1;
              ok = false;
              break;
            }
            uint8_t* sa = ring + (size_t)slot * STAGE;
            mbar_expect_tx(&full_bar[slot], STAGE);
            const int c = (int)(col0 + (int64_t)t * KB);
            tma_load(sa, mapX, &full_bar[slot], c, row0);
            tma_load(sa + STAGE / 2, mapX, &full_bar[slot], c + 64, row0);
          }
        }
      }
      // let the copies already issued land before the CTA can leave
      mbar_wait(&vfull_bar, 0u, err);
      for (int64_t u = i - nst < 0 ? 0 : i - nst; u < i; ++u)
        mbar_wait(&full_bar[u % nst], (uint32_t)(u / nst) & 1u, err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // --------------------------------------------------------- MMA issue
      const uint32_t idxv = d.f16 ? IDESC_XV_H : IDESC_XV_BF;
      const uint32_t idxt = d.f16 ? IDESC_XT_H : IDESC_XT_BF;
      const uint32_t vh = saddr(vres), vl = saddr(vres + (size_t)S * RP * 2);
      const uint32_t uh = saddr(ubuf), ul = saddr(ubuf + (size_t)TILE * RP * 2);
      bool ok = fwait(&vfull_bar, 0u, err, false);
      int64_t i = 0;
      for (int s = 0; ok && s < npan + LAG; ++s) {
        if (s < npan) {
          const int b = s % NACC;
          if (!fwait(&acce_bar[b], ((uint32_t)(s / NACC) & 1u) ^ 1u, err, false)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t dcol = tmem + (uint32_t)(b * RP);
          for (int t = 0; t < T; ++t, ++i) {
            const int slot = (int)(i % nst);
            if (!fwait(&full_bar[slot], (uint32_t)(i / nst) & 1u, err, false)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = saddr(ring + (size_t)slot * STAGE);
#pragma unroll
            for (int kk = 0; kk < KB / 16; ++kk) {
              const uint32_t aoff = (uint32_t)(kk / 4) * (STAGE / 2) + (uint32_t)(kk % 4) * 32;
              const uint32_t boff = (uint32_t)(2 * t + kk / 4) * ATOM + (uint32_t)(kk % 4) * 32;
              const uint64_t da = sdesc(a0 + aoff, 16, 1024);
              mma_f16kind(dcol, da, sdesc(vh + boff, 16, 1024), idxv, (t > 0 || kk > 0) ? 1u : 0u);
              mma_f16kind(dcol, da, sdesc(vl + boff, 16, 1024), idxv, 1u);
            }
            mma_commit(&empty_bar[slot]);
          }
          if (!ok) break;
          mma_commit(&accf_bar[b]);
        }
        const int pj = s - LAG;
        if (pj >= 0 && pj < npan) {
          if (!fwait(&uready_bar[pj & 1], (uint32_t)(pj >> 1) & 1u, err, true)) {
            ok = false;
            break;
          }
          stamp(sst, stamping, pj, 6);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          for (int t = 0; t < T; ++t, ++i) {
            const int slot = (int)(i % nst);
            if (!fwait(&full_bar[slot], (uint32_t)(i / nst) & 1u, err, false)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = saddr(ring + (size_t)slot * STAGE);
            const uint32_t dt = tmem + (uint32_t)((NACC + t) * RP);
#pragma unroll
            for (int kk = 0; kk < KB / 16; ++kk) {
              // A = X stage read MN-major (16 panel rows = 2048 bytes per K
              // step, the two 64-column atoms 16 KB apart); B = U panel pair
              const uint64_t da = sdesc(a0 + kk * 2048, STAGE / 2, 1024);
              const uint32_t boff = (uint32_t)(kk / 4) * ATOM + (uint32_t)(kk % 4) * 32;
              mma_f16kind(dt, da, sdesc(uh + boff, 16, 1024), idxt, (pj > 0 || kk > 0) ? 1u : 0u);
              mma_f16kind(dt, da, sdesc(ul + boff, 16, 1024), idxt, 1u);
            }
            mma_commit(&empty_bar[slot]);
          }
          if (!ok) break;
          // the U panel buffer of every CTA may take the next panel once
          // these MMAs (and every other CTA's) have read it
          mma_commit_multicast(&ufree_bar[pj & 1], cmask);
          stamp(sst, stamping, pj, 7);
        }
      }
      if (!ok) aborted = 1;
      mma_commit(&drain_bar);
    }
  } else if (warp >= 6) {
    // ------------------------------------------------ writers (warps 6-7)
    // The new rows of U of each panel, from the epilogue's buffer: U (FP32,
    // m x r) and the U^T pair (for the X_lo pass), 16-byte chunks of 8 rows.
    const int wt = threadIdx.x - 192;       // 0..63
    bool ok = true;
    for (int pi = 0; pi < npan; ++pi) {
      const int p = q + pi * Q, par = pi & 1;
      if (ok && !fwait(&wready_bar[par], (uint32_t)(pi >> 1) & 1u, err, false)) ok = false;
      const float* ur = urow + (size_t)par * Rc * RP;
      const int64_t row0 = (int64_t)p * TILE + (int64_t)j * Rc;
      for (int e = wt; ok && e < Rc * r; e += 64) {
        const int rr = e / r, l = e % r;
        if (row0 + rr < m) d.U[(row0 + rr) * r + l] = ur[rr * RP + l];
      }
      const int nchunk = r * 2 * (Rc / 8);
      for (int ch = wt; ok && ch < nchunk; ch += 64) {
        const int c = ch % r, h = (ch / r) & 1, g = ch / (2 * r);
        const int64_t i0 = row0 + 8 * g;
        if (i0 >= m) continue;
        uint32_t w[4];
#pragma unroll
        for (int t2 = 0; t2 < 4; ++t2) {
          const float x0 = ur[(8 * g + 2 * t2) * RP + c], x1 = ur[(8 * g + 2 * t2 + 1) * RP + c];
          uint16_t b0 = to16b(x0, d.f16), b1 = to16b(x1, d.f16);
          if (h) {
            b0 = to16b(x0 - from16b(b0, d.f16), d.f16);
            b1 = to16b(x1 - from16b(b1, d.f16), d.f16);
          }
          w[t2] = (uint32_t)b0 | ((uint32_t)b1 << 16);
        }
        uint8_t* dst = reinterpret_cast<uint8_t*>(h ? d.utl : d.uth) + ((int64_t)c * d.ldm + i0) * 2;
        *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
      }
      asm volatile("bar.sync 2, 64;" ::: "memory");
      if (wt == 0) mbar_arrive(&wdone_bar[par]);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int et = threadIdx.x - 64;        // 0..127
    const int quarter = warp & 3;           // TMEM lanes 32 quarter .. + 31
    const int lrow = quarter * 32 + lane;   // accumulator row of this thread
    const int rho = et / 8, sub = et % 8;   // HALS: row rho of my R rows, lane sub of 8
    const bool hals_thread = rho < Rc;
    // Gram of this CTA's new rows, entries idx = et + 128 w (FP32 sums)
    constexpr int GW = RP * RP / 128;
    float gacc[GW];
#pragma unroll
    for (int w = 0; w < GW; ++w) gacc[w] = 0.f;
    bool ok = true;
    float u_nx[4 * NV], cv_nx[4 * NV];     // the next panel's row of U and X_lo V
    {
      const int64_t g0 = (int64_t)q * TILE + (int64_t)j * Rc + rho;
      const bool l0 = hals_thread && npan > 0 && g0 < m;
#pragma unroll
      for (int e = 0; e < 4 * NV; ++e) {
        const int l = 32 * (e / 4) + 4 * sub + (e % 4);
        u_nx[e] = (l0 && l < r) ? __ldcg(d.U + g0 * r + l) : 0.f;
        cv_nx[e] = (l0 && l < r && d.cv) ? __ldcg(d.cv + g0 * r + l) : 0.f;
      }
    }
    for (int pi = 0; pi < npan; ++pi) {
      const int p = q + pi * Q;
      const int b = pi % NACC, par = pi & 1;
      const uint32_t ph2 = (uint32_t)(pi >> 1) & 1u;
      // 1. the panel's X V partial of my slice: tensor memory -> xstg
      if (ok && !fwait(&accf_bar[b], (uint32_t)(pi / NACC) & 1u, err, false)) ok = false;
      if (et == 0) stamp(sst, stamping, pi, 0);
      const int k = (int)j * Rc + rho;                 // panel row
      const int64_t gi = (int64_t)p * TILE + k;        // row of X and U
      const bool live = hals_thread && gi < m;
      // this thread's row of U and of the X_lo V term were requested one
      // panel ahead (global loads wait behind the X stream); take them and
      // request the next panel's
      float u[4 * NV], cvr[4 * NV];
#pragma unroll
      for (int e = 0; e < 4 * NV; ++e) {
        u[e] = u_nx[e];
        cvr[e] = cv_nx[e];
      }
      {
        const int64_t gn = (int64_t)(p + Q) * TILE + k;
        const bool ln = hals_thread && pi + 1 < npan && gn < m;
#pragma unroll
        for (int e = 0; e < 4 * NV; ++e) {
          const int l = 32 * (e / 4) + 4 * sub + (e % 4);
          u_nx[e] = (ln && l < r) ? __ldcg(d.U + gn * r + l) : 0.f;
          cv_nx[e] = (ln && l < r && d.cv) ? __ldcg(d.cv + gn * r + l) : 0.f;
        }
      }
      if (ok && pi > 0 && !fwait(&consumed_bar[(pi - 1) & 1], (uint32_t)((pi - 1) >> 1) & 1u, err, true))
        ok = false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // (tcgen05.ld is warp-collective: the whole warp loads, or none of it)
      if (__all_sync(0xffffffffu, ok)) {
#pragma unroll
        for (int c0 = 0; c0 < RP; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * RP + c0), v);
#pragma unroll
          for (int u = 0; u < 16; u += 4)
            *reinterpret_cast<float4*>(&xstg[lrow * XLD + c0 + u]) =
                make_float4(v[u], v[u + 1], v[u + 2], v[u + 3]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (et == 0) mbar_arrive(&acce_bar[b]);   // accumulator b free for panel pi + NACC
      // One remote arrival per thread (thread c signals CTA c): a release
      // arrival waits for its own round trip, so C of them from one thread
      // would take C round trips in a row.
      if (et < C && ok) mbar_arrive_remote(peer_addr(saddr(&staged_bar[par]), (uint32_t)et));
      // 2. my rows of the panel: the C partials summed in CTA order
      if (ok && !fwait(&staged_bar[par], ph2, err, true)) ok = false;
      if (et == 0) stamp(sst, stamping, pi, 1);
      float a[4 * NV];
#pragma unroll
      for (int e = 0; e < 4 * NV; ++e) a[e] = 0.f;
      if (ok && hals_thread) {
        const uint32_t rbase = saddr(&xstg[k * XLD]);
        for (int c = 0; c < C; ++c) {
          const uint32_t pb = peer_addr(rbase, (uint32_t)c);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const float4 x = ld_cluster_v4(pb + (uint32_t)((32 * v + 4 * sub) * 4));
            a[4 * v] += x.x;
            a[4 * v + 1] += x.y;
            a[4 * v + 2] += x.z;
            a[4 * v + 3] += x.w;
          }
        }
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (et == 0) stamp(sst, stamping, pi, 2);
      if (et < C && ok) mbar_arrive_remote(peer_addr(saddr(&consumed_bar[par]), (uint32_t)et));
      // 3. HALS on the row: u_l <- max(0, u_l + (a_l - u . G_:l) / G_ll), l in order
      float qv[4 * NV];
#pragma unroll
      for (int e = 0; e < 4 * NV; ++e) a[e] += cvr[e];
      // q = a - u G, with u gathered across the row's eight lanes
#pragma unroll
      for (int e = 0; e < 4 * NV; ++e) qv[e] = a[e];
#pragma unroll
      for (int o = 0; o < 8; ++o) {
#pragma unroll
        for (int e2 = 0; e2 < 4 * NV; ++e2) {
          const int c = 32 * (e2 / 4) + 4 * o + (e2 % 4);
          const float uc = __shfl_sync(0xffffffffu, u[e2], (lane & ~7) | o);
#pragma unroll
          for (int e = 0; e < 4 * NV; ++e) {
            const int l = 32 * (e / 4) + 4 * sub + (e % 4);
            qv[e] = fmaf(-uc, Gs[c * RP + l], qv[e]);
          }
        }
      }
#pragma unroll
      for (int jc = 0; jc < RP; ++jc) {
        const int own = (jc % 32) / 4, ee = (jc / 32) * 4 + jc % 4;
        const float gi_j = ginv[jc];
        float dl = 0.f;
        if (sub == own && gi_j > 0.f && jc < r) {
          float v = fmaf(qv[ee], gi_j, u[ee]);
          v = v > 0.f ? v : 0.f;
          dl = v - u[ee];
          u[ee] = v;
        }
        dl = __shfl_sync(0xffffffffu, dl, (lane & ~7) | own);
#pragma unroll
        for (int e = 0; e < 4 * NV; ++e) {
          const int l = 32 * (e / 4) + 4 * sub + (e % 4);
          qv[e] = fmaf(-dl, Gs[jc * RP + l], qv[e]);
        }
      }
      if (et == 0) stamp(sst, stamping, pi, 3);
      // the writer warps have written out this buffer's rows of panel pi - 2
      float* const ur = urow + (size_t)par * Rc * RP;
      if (ok && pi >= 2 && !fwait(&wdone_bar[par], (uint32_t)((pi - 2) >> 1) & 1u, err, false))
        ok = false;
      if (hals_thread) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          float4 w4 = make_float4(live ? u[4 * v] : 0.f, live ? u[4 * v + 1] : 0.f,
                                  live ? u[4 * v + 2] : 0.f, live ? u[4 * v + 3] : 0.f);
          *reinterpret_cast<float4*>(&ur[rho * RP + 32 * v + 4 * sub]) = w4;
        }
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      // the rows go to global memory through the writer warps (warps 6-7), so
      // that no global store precedes this CTA's cluster-scope releases
      if (et == 0) mbar_arrive(&wready_bar[par]);
      // 4. Gram of the new rows
#pragma unroll
      for (int w = 0; w < GW; ++w) {
        const int idx = et + 128 * w, ga = idx / RP, gb = idx % RP;
        float s = gacc[w];
        for (int rr = 0; rr < Rc; ++rr) s = fmaf(ur[rr * RP + ga], ur[rr * RP + gb], s);
        gacc[w] = s;
      }
      // 5. push my rows of U into every CTA's panel buffer (16-bit pair, one
      // 16-byte chunk = 8 consecutive panel rows of one column)
      if (ok && pi > 0 && !fwait(&ufree_bar[(pi - 1) & 1], (uint32_t)((pi - 1) >> 1) & 1u, err, true))
        ok = false;
      if (et == 0) stamp(sst, stamping, pi, 4);
      const int nchunk = RP * 2 * (Rc / 8);
      for (int ch = et; ok && ch < nchunk; ch += 128) {
        const int c = ch % RP, h = (ch / RP) & 1, g = ch / (2 * RP);
        const int k0 = (int)j * Rc + 8 * g;
        uint32_t w[4];
#pragma unroll
        for (int t2 = 0; t2 < 4; ++t2) {
          const float x0 = ur[(8 * g + 2 * t2) * RP + c], x1 = ur[(8 * g + 2 * t2 + 1) * RP + c];
          uint16_t b0 = to16b(x0, d.f16), b1 = to16b(x1, d.f16);
          if (h) {
            b0 = to16b(x0 - from16b(b0, d.f16), d.f16);
            b1 = to16b(x1 - from16b(b1, d.f16), d.f16);
          }
          w[t2] = (uint32_t)b0 | ((uint32_t)b1 << 16);
        }
        const uint4 cv4 = make_uint4(w[0], w[1], w[2], w[3]);
        const uint32_t off = (uint32_t)h * (TILE * RP * 2) + (uint32_t)(k0 / 64) * ATOM +
                             (uint32_t)c * 128 + ((((uint32_t)(k0 % 64) / 8) ^ (uint32_t)(c & 7)) << 4);
        const uint32_t local = saddr(ubuf + off);
        for (int cc = 0; cc < C; ++cc) st_cluster_v4(peer_addr(local, (uint32_t)cc), cv4);
      }
      asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (et < C && ok) mbar_arrive_remote(peer_addr(saddr(&uready_bar[par]), (uint32_t)et));
      if (et == 0) stamp(sst, stamping, pi, 5);
      // (no early exit: every epilogue thread meets every named barrier of
      // every panel; after a failed wait a thread only skips its work)
    }
    if (!ok) aborted = 1;
    // ---- the CTA's Gram partial (FP64)
    const int rr2 = r * r;
#pragma unroll
    for (int w = 0; w < GW; ++w) {
      const int idx = et + 128 * w, ga = idx / RP, gb = idx % RP;
      if (ga < r && gb < r) d.gpart[(int64_t)blockIdx.x * rr2 + ga * r + gb] = (double)gacc[w];
    }
    // ---- X^T U of the slice: tensor memory -> the cluster's partial
    const bool drained = fwait(&drain_bar, 0u, err, false);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__all_sync(0xffffffffu, drained && ok && !*(volatile int*)&aborted)) {
      for (int t = 0; t < T; ++t) {
        const int64_t row = (int64_t)j * S + (int64_t)t * TILE + lrow;
        float* dst = d.xtu + ((int64_t)q * n + row) * r;
#pragma unroll
        for (int c0 = 0; c0 < RP; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((NACC + t) * RP + c0), v);
          if (row < n) {
#pragma unroll
            for (int u2 = 0; u2 < 16; ++u2)
              if (c0 + u2 < r) dst[c0 + u2] = npan > 0 ? v[u2] : 0.f;
          }
        }
      }
    }
    // ---- U^T U: the last CTA of the launch sums the partials in CTA order
    __threadfence();
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (et == 0) {
      const int old = atomicAdd(d.counter, 1);
      last_cta = old == (int)gridDim.x - 1;
      if (last_cta) *d.counter = 0;
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (last_cta) {
      __threadfence();
      const int G = (int)gridDim.x;
      for (int e = et; e < rr2; e += 128) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int bb = 0;
        for (; bb + 4 <= G; bb += 4) {
          s0 += __ldcg(&d.gpart[(int64_t)bb * rr2 + e]);
          s1 += __ldcg(&d.gpart[(int64_t)(bb + 1) * rr2 + e]);
          s2 += __ldcg(&d.gpart[(int64_t)(bb + 2) * rr2 + e]);
          s3 += __ldcg(&d.gpart[(int64_t)(bb + 3) * rr2 + e]);
        }
        for (; bb < G; ++bb) s0 += __ldcg(&d.gpart[(int64_t)bb * rr2 + e]);
        d.Gu[e] = (s0 + s1) + (s2 + s3);
      }
    }
  }
  if (threadIdx.x == 64) stamp(sst, stamping, STAMP_PANELS, 1);
  __syncthreads();
  if (stamping)
    for (int e = threadIdx.x; e < (STAMP_PANELS + 1) * 8; e += THREADS)
      d.stamps[(int64_t)blockIdx.x * (STAMP_PANELS + 1) * 8 + e] = sst[e];
  // every MMA of the CTA has completed, and no peer still touches this CTA's
  // shared memory, before tensor memory is freed and the CTA leaves
  mbar_wait(&drain_bar, 0u, err);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  cluster_sync_all();
  if (warp == 1) {
    const uint32_t cols = tmem_cols <= 32 ? 32 : tmem_cols <= 64 ? 64 : tmem_cols <= 128 ? 128
                          : tmem_cols <= 256 ? 256 : 512;
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols)
                 : "memory");
  }
}

}  // namespace fz

// ------------------------------------------------------------------- host
template <int RP>
static cudaError_t fused_launch_rp(const FusedDesc* fd, const FusedPlan& pl, cudaStream_t s) {
  auto kern = fz::fused_hals_kernel<RP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  if (pl.C > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)(pl.Q * pl.C));
  cfg.blockDim = dim3(fz::THREADS);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)pl.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, fd, pl.nst);
}

template <int RP>
static int fused_max_clusters(const FusedPlan& pl) {
  auto kern = fz::fused_hals_kernel<RP>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (pl.C > 8 &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)pl.C);
  cfg.blockDim = dim3(fz::THREADS);
  cfg.dynamicSmemBytes = pl.smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)pl.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nc;
}

// Plan of the fused kernel for an m x n problem at rank pad rp: the cluster
// size (16, else 8), the slice width, the ring depth and the clusters; ok =
// false when tensor memory, shared memory or the cluster shape do not fit
// (the two-pass sweeps are used then).
FusedPlan fused_plan(int64_t m, int64_t n, int rp) {
  FusedPlan pl;
  memset(&pl, 0, sizeof(pl));
  if (rp != 32 && rp != 64) return pl;
  const int64_t npanels = (m + fz::TILE - 1) / fz::TILE;
  if (npanels > 0x7fffffff || n > 0x7fffffffLL) return pl;
  const size_t budget = 227 * 1024 - 4096;   // less static shared memory (barriers, stamps)
  int order[2] = {16, 8};
  if (const char* e = getenv("ENMF_FUSED_CLUSTER")) {   // diagnostics: force 8 or 16
    if (atoi(e) == 8) {
      order[0] = 8;
      order[1] = 8;
    }
  }
  for (int C : order) {
    const int64_t S = ((n + (int64_t)C * fz::KB - 1) / ((int64_t)C * fz::KB)) * fz::KB;
    const int T = (int)(S / fz::TILE);
    if ((fz::NACC + T) * rp > 512) continue;
    int nst = 0;
    for (int st = fz::MAX_STAGES; st >= 2; --st)
      if (fz::smem_plan(rp, (int)S, C, st).total <= budget) {
        nst = st;
        break;
      }
    if (nst < 2) continue;
    FusedPlan t = pl;
    t.C = C;
    t.S = (int)S;
    t.T = T;
    t.nst = nst;
    t.smem = fz::smem_plan(rp, (int)S, C, nst).total;
    t.npanels = (int)npanels;
    const int nc = rp == 32 ? fused_max_clusters<32>(t) : fused_max_clusters<64>(t);
    if (nc < 1) continue;
    t.Q = (int)(npanels < nc ? npanels : nc);
    t.ok = 1;
    return t;
  }
  return pl;
}

cudaError_t launch_fused(const FusedDesc* fd, const FusedPlan& pl, int rp, cudaStream_t s) {
  note_launch(1);
  return rp == 32 ? fused_launch_rp<32>(fd, pl, s) : fused_launch_rp<64>(fd, pl, s);
}

}  // namespace enmf
