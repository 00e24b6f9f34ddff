// Tensor-core sweeps over a BF16 copy of X for the reduced-precision form:
//   X V   (A = X tile, K-major)       and
//   X^T U (A = X tile read MN-major),
// each on the 5th-generation tensor cores (tcgen05.mma, kind::f16, BF16
// operands, FP32 accumulator in tensor memory).  X tiles are streamed by TMA
// (cp.async.bulk.tensor, 128-byte swizzle) through a multi-stage shared-memory
// ring; one elected thread issues the TMA copies, one issues the MMAs, and
// tcgen05.commit releases each stage back to the producer.
//
// The factor operand is held as a BF16 pair F = F_hi + F_lo (F_hi = bf16(F),
// F_lo = bf16(F - F_hi)), transposed so that the reduction index is
// contiguous (K-major B); two MMAs per K step accumulate X F_hi + X F_lo, which
// keeps about 16 bits of the FP32 factor.  X itself is BF16 (X_hi); the
// remainder X_lo = bf16(X - X_hi) is applied every few iterations by the
// same kernels (the correction of the precision form).
//
// Persistent, stream-K schedule: one CTA per SM, each owning an equal
// contiguous range of the (output tile, k-block) space; two tensor-memory
// accumulators let the epilogue of one tile overlap the MMAs of the next.
// The sweep reads X once per product, so at small rank it is bound by HBM
// bandwidth: algorithmic bytes per sweep = m n * 2.
//
// FP8 stream form (XQ): X_hi is held as e4m3 codes with one power-of-two
// scale 2^k per 128 x 128 tile of X.  TMA streams the one-byte codes (half
// the bytes of BF16); four converter warps rebuild each tile in shared
// memory as the exact BF16 values q 2^k, in the same swizzled layout a TMA
// copy of a BF16 tile would have, and the MMA path is the BF16 one.  The
// factor tiles have a ring of their own, filled by the producer ahead of the
// MMAs; the factor's hi and lo rows sit side by side so that one MMA with
// N = 2 RP covers both (the X tile is read once per K step).  Algorithmic
// bytes per sweep = m n.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <math.h>

#include "internal.h"
#include "tail.cuh"
#include "tc_ptx.cuh"

namespace enmf {

namespace tc {

constexpr int TILE = 128;     // output rows per CTA (UMMA M)
constexpr int KB_XV = 128;    // reduction columns per stage, X V (two 64-column boxes)
constexpr int KB_XT = 128;    // reduction rows per stage, X^T U
constexpr int THREADS = 192;  // warp 0 TMA producer, warp 1 MMA issuer, warps 2-5 epilogue
constexpr int THREADS_XQ = 320;  // the same, plus warps 6-9 converting FP8 tiles to BF16
constexpr int NCW = 4;           // converter warps of the FP8 form
constexpr uint32_t Q_BYTES = 128 * 128;  // one FP8 X tile (128 x 128 codes)
constexpr int MAX_GRID = 256;  // CTAs of the persistent sweep at most

// Work split (stream-K): the work of all problems, each problem's (tile,
// k-block) units tile-major and the problems one after another, is cut into
// G contiguous ranges of equal length, one per CTA.  A CTA walks its range as
// segments of consecutive k-blocks of one tile; a segment that covers a whole
// tile writes the result directly, the (at most two) partial segments at the
// ends of a range write FP32 partial slots; the last CTA to finish a cut tile
// (a per-tile arrival counter) sums its slots in CTA order.  Problem
// boundaries are tile boundaries, so this holds across problems.
__host__ __device__ __forceinline__ int64_t sk_begin(int64_t c, int64_t W, int64_t G) {
  return (c * W) / G;
}

// The problem holding global unit w (descriptors in work order, np >= 1).
__device__ __forceinline__ int prob_find(const SweepProb* probs, int np, int64_t w) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (probs[mid].w_begin <= w) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// A CTA's view of the problem its current units belong to.
template <int KB>
struct ProbView {
  const SweepProb* d;
  int64_t wb, we, nkb;   // first unit, one past the last unit, k-blocks per tile
  __device__ __forceinline__ void load(const SweepProb* probs, int np, int p, int64_t W) {
    d = probs + p;
    wb = d->w_begin;
    we = p + 1 < np ? probs[p + 1].w_begin : W;
    nkb = (d->red + KB - 1) / KB;
  }
};

// MODE 0: C = X V (rows_out = m, reduction over n; A = X tile, K-major).
// MODE 1: C = X^T U (rows_out = n, reduction over m; A = X tile, MN-major).
// Per problem (SweepProb): X map, the factor transposed as a BF16 pair
// (mapBh / mapBl, RP x red), out (rows_out x r, FP32) receiving whole tiles
// (+ corr when given).  part [G][2][TILE][RP] receives the partial segments.
// XQ: the FP8 stream form (X tiles as e4m3 codes with per-tile exponents,
// see the file comment); qstages / bstages = depths of its FP8 tile ring and
// of its factor-tile ring.
template <int MODE, int RP, bool XQ = false>
__global__ void __launch_bounds__(XQ ? THREADS_XQ : THREADS, 1)
sweep_tc_kernel(const SweepProb* __restrict__ probs, int np, int64_t W, int stages,
                float* __restrict__ part, int* __restrict__ counters, int fixup, int* err,
                int qstages, int bstages) {
  constexpr int KB = MODE == 0 ? KB_XV : KB_XT;
  constexpr uint32_t A_BYTES = TILE * KB * 2;                 // 16 KB or 32 KB
  constexpr uint32_t B_BYTES = RP * KB * 2;                   // one of hi / lo
  constexpr uint32_t STAGE = A_BYTES + 2 * B_BYTES;
  // non-FP8 forms: X V's X tile is KB / 64 boxes of 64 columns side by side;
  // the factor's hi and lo tiles are KB / 64 boxes of 64 K elements each
  constexpr int NBOX = KB / 64;
  constexpr uint32_t BOXA = TILE * 64 * 2;
  constexpr uint32_t BOXB = RP * 64 * 2;
  static_assert(KB % 64 == 0 && (MODE == 0 || KB == 128) && (!XQ || KB == 128),
                "X^T U and the FP8 form take 128-row stages");
  // XQ: the factor tiles live in a ring of their own, so a stage is A only
  constexpr uint32_t ASTAGE = XQ ? A_BYTES : STAGE;
  constexpr uint32_t BSLOT = 2 * B_BYTES;   // [hi | lo | hi | lo] boxes of one unit
  constexpr uint32_t IDESC_BF16 = idesc_f16kind(TILE, RP, MODE, 0);
  constexpr uint32_t IDESC_F16 = idesc_f16kind(TILE, RP, MODE, 1);
  // XQ: one MMA over [hi | lo] rows of the factor (N = 2 RP) into an
  // accumulator of 2 RP columns (hi and lo products summed in the epilogue)
  constexpr uint32_t IDESC_XQ = idesc_f16kind(TILE, 2 * RP, MODE, 0);
  constexpr uint32_t ACC_COLS = XQ ? 2 * RP : RP;
  constexpr uint32_t TMEM_COLS =
      XQ ? (RP <= 16 ? 64 : (RP <= 32 ? 128 : 256)) : (RP <= 32 ? 64 : 128);  // two accumulators
  constexpr int QB = XQ ? 8 : 1;

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[8];
  __shared__ __align__(8) uint64_t empty_bar[8];
  __shared__ __align__(8) uint64_t bfull_bar[QB];    // XQ: factor tiles of a unit landed
  __shared__ __align__(8) uint64_t bempty_bar[QB];   // XQ: factor slot consumed by the MMAs
  __shared__ __align__(8) uint64_t qfull_bar[QB];    // XQ: FP8 tile landed
  __shared__ __align__(8) uint64_t qempty_bar[QB];   // XQ: FP8 tile consumed
  __shared__ __align__(8) uint64_t accf_bar[2];
  __shared__ __align__(8) uint64_t acce_bar[2];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int aborted;
  __shared__ int last_cta;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  // XQ: [A stages][factor ring][FP8 ring][epilogue staging]
  uint8_t* const bring = smem + (size_t)stages * ASTAGE;
  uint8_t* const qring = bring + (XQ ? (size_t)bstages * BSLOT : 0);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t G = gridDim.x;
  const int64_t w0 = sk_begin(blockIdx.x, W, G), w1 = sk_begin(blockIdx.x + 1, W, G);
  const int p0 = w0 < w1 ? prob_find(probs, np, w0) : 0;

  int64_t pre = 0;   // (thread 0) units whose X tiles were requested in the prologue
  if (threadIdx.x == 0) {
    if (w0 < w1) {
      prefetch_map(reinterpret_cast<const CUtensorMap*>(probs[p0].mapX));
      prefetch_map(reinterpret_cast<const CUtensorMap*>(probs[p0].mapBh));
      prefetch_map(reinterpret_cast<const CUtensorMap*>(probs[p0].mapBl));
    }
    for (int s = 0; s < stages; ++s) {
      // XQ: a stage's X tile is complete when every converter warp arrived
      mbar_init(&full_bar[s], XQ ? NCW : 1);
      mbar_init(&empty_bar[s], 1);
    }
    if constexpr (XQ) {
      for (int q = 0; q < qstages; ++q) {
        mbar_init(&qfull_bar[q], 1);
        mbar_init(&qempty_bar[q], NCW);
      }
      for (int b = 0; b < bstages; ++b) {
        mbar_init(&bfull_bar[b], 1);
        mbar_init(&bempty_bar[b], 1);
      }
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], 4);
    }
    mbar_init(&drain_bar, 1);
    aborted = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // Thread 0 is the producer.  The X tiles of the first `stages` units (of
    // the first problem) are requested now, before the tensor-memory
    // allocation and before the wait for the previous kernel; their factor
    // tiles after that wait (the stage's transaction count covers both).
    // The ring's first pass needs no empty-slot wait.
    if constexpr (!XQ) {
      if (w0 < w1) {
        ProbView<KB> pv;
        pv.load(probs, np, p0, W);
        const uint64_t xpol = l2_policy(pv.d->l2hint);
        const CUtensorMap* mapX = reinterpret_cast<const CUtensorMap*>(pv.d->mapX);
        for (int64_t w = w0; w < w1 && w < pv.we && pre < stages; ++w, ++pre) {
          const int64_t lw = w - pv.wb;
          const int t0 = (int)((lw / pv.nkb) * TILE);
          const int k0 = (int)((lw % pv.nkb) * KB);
          uint8_t* sa = smem + (size_t)pre * STAGE;
          mbar_expect_tx(&full_bar[pre], STAGE);
          if (MODE == 0) {
#pragma unroll
            for (int bx = 0; bx < NBOX; ++bx)
              tma_load_hint(sa + bx * BOXA, mapX, &full_bar[pre], k0 + 64 * bx, t0, xpol);
          } else {
            tma_load_hint(sa, mapX, &full_bar[pre], t0, k0, xpol);
            tma_load_hint(sa + A_BYTES / 2, mapX, &full_bar[pre], t0 + 64, k0, xpol);
          }
        }
      }
    }
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // Launched as a programmatic dependent (of the half step that wrote the
  // factor), the CTA gets here while that kernel may still run: only X, which
  // no kernel of the iteration writes, is read before griddep_wait().
  griddep_launch();

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------- producer
      int p = p0;
      ProbView<KB> pv;
      pv.load(probs, np, p, W);
      int64_t i = 0;
      int64_t q_issued = 0, b_issued = 0;   // XQ: units whose copies were requested
      uint64_t xpol = l2_policy(pv.d->l2hint);
      griddep_wait();
      // (the prefetched units always get their factor tiles, so that every
      // stage with copies in flight completes)
      for (int64_t w = w0; w < w1 && (i < pre || !*(volatile int*)&aborted); ++w, ++i) {
        if (w >= pv.we) {
          pv.load(probs, np, ++p, W);
          xpol = l2_policy(pv.d->l2hint);
          prefetch_map(reinterpret_cast<const CUtensorMap*>(pv.d->mapX));
          prefetch_map(reinterpret_cast<const CUtensorMap*>(pv.d->mapBh));
          prefetch_map(reinterpret_cast<const CUtensorMap*>(pv.d->mapBl));
        }
        const CUtensorMap* mapX = reinterpret_cast<const CUtensorMap*>(pv.d->mapX);
        if constexpr (XQ) {
          // one 128 x 128 box of codes per unit into the FP8 ring, then the
          // unit's factor tiles into the factor ring (each ring runs ahead of
          // its consumer by its depth)
          const int q = (int)(i % qstages);
          const uint32_t qph = (uint32_t)(i / qstages) & 1u;
          if (!mbar_wait(&qempty_bar[q], qph ^ 1u, err)) {
            aborted = 1;
            break;
          }
          const int64_t lw = w - pv.wb;
          const int t0 = (int)((lw / pv.nkb) * TILE);
          const int k0 = (int)((lw % pv.nkb) * KB);
          uint8_t* sq = qring + (size_t)q * Q_BYTES;
          mbar_expect_tx(&qfull_bar[q], Q_BYTES);
          if (MODE == 0) tma_load_hint(sq, mapX, &qfull_bar[q], k0, t0, xpol);
          else tma_load_hint(sq, mapX, &qfull_bar[q], t0, k0, xpol);
          q_issued = i + 1;
          const int bs = (int)(i % bstages);
          const uint32_t bph = (uint32_t)(i / bstages) & 1u;
          if (!mbar_wait(&bempty_bar[bs], bph ^ 1u, err)) {
            aborted = 1;
            break;
          }
          const CUtensorMap* mapBh = reinterpret_cast<const CUtensorMap*>(pv.d->mapBh);
          const CUtensorMap* mapBl = reinterpret_cast<const CUtensorMap*>(pv.d->mapBl);
          uint8_t* sb = bring + (size_t)bs * BSLOT;
          mbar_expect_tx(&bfull_bar[bs], BSLOT);
          tma_load(sb, mapBh, &bfull_bar[bs], k0, 0);
          tma_load(sb + B_BYTES / 2, mapBl, &bfull_bar[bs], k0, 0);
          tma_load(sb + B_BYTES, mapBh, &bfull_bar[bs], k0 + 64, 0);
          tma_load(sb + 3 * B_BYTES / 2, mapBl, &bfull_bar[bs], k0 + 64, 0);
          b_issued = i + 1;
          continue;
        }
        const CUtensorMap* mapBh = reinterpret_cast<const CUtensorMap*>(pv.d->mapBh);
        const CUtensorMap* mapBl = reinterpret_cast<const CUtensorMap*>(pv.d->mapBl);
        const int s = (int)(i % stages);
        const uint32_t ph = (uint32_t)(i / stages) & 1u;
        if (i >= pre && !mbar_wait(&empty_bar[s], ph ^ 1u, err)) {
          aborted = 1;
          break;
        }
        const int64_t lw = w - pv.wb;
        const int64_t tile = lw / pv.nkb, kb = lw % pv.nkb;
        const int t0 = (int)(tile * TILE);
        const int k0 = (int)(kb * KB);
        uint8_t* sa = smem + (size_t)s * STAGE;
        uint8_t* sbh = sa + A_BYTES;
        uint8_t* sbl = sbh + B_BYTES;
        if (i >= pre) {
          mbar_expect_tx(&full_bar[s], STAGE);
          if (MODE == 0) {
            // adjacent 64-column boxes: KB * 2 contiguous bytes of each X row
#pragma unroll
            for (int bx = 0; bx < NBOX; ++bx)
              tma_load_hint(sa + bx * BOXA, mapX, &full_bar[s], k0 + 64 * bx, t0, xpol);
          } else {
            tma_load_hint(sa, mapX, &full_bar[s], t0, k0, xpol);
            tma_load_hint(sa + A_BYTES / 2, mapX, &full_bar[s], t0 + 64, k0, xpol);
          }
        }
#pragma unroll
        for (int bx = 0; bx < NBOX; ++bx) {
          tma_load(sbh + bx * BOXB, mapBh, &full_bar[s], k0 + 64 * bx, 0);
          tma_load(sbl + bx * BOXB, mapBl, &full_bar[s], k0 + 64 * bx, 0);
        }
      }
      if (aborted) {
        // let copies already issued land before the CTA can exit
        const int64_t issued = i;
        if constexpr (XQ) {
          for (int64_t q = q_issued - qstages < 0 ? 0 : q_issued - qstages; q < q_issued; ++q)
            mbar_wait(&qfull_bar[q % qstages], (uint32_t)(q / qstages) & 1u, err);
          for (int64_t u = b_issued - bstages < 0 ? 0 : b_issued - bstages; u < b_issued; ++u)
            mbar_wait(&bfull_bar[u % bstages], (uint32_t)(u / bstages) & 1u, err);
        } else {
          for (int64_t q = issued - stages < 0 ? 0 : issued - stages; q < issued; ++q)
            mbar_wait(&full_bar[q % stages], (uint32_t)(q / stages) & 1u, err);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // --------------------------------------------------------- MMA issue
      griddep_wait();   // (its bounded waits start once the factor can land)
      int p = p0;
      ProbView<KB> pv;
      pv.load(probs, np, p, W);
      int64_t i = 0;
      int64_t seg = 0;
      for (int64_t w = w0; w < w1 && !*(volatile int*)&aborted; ++seg) {
        if (w >= pv.we) pv.load(probs, np, ++p, W);
        const int64_t tile = (w - pv.wb) / pv.nkb;
        const int64_t wend = min(w1, pv.wb + (tile + 1) * pv.nkb);
        const int b = (int)(seg & 1);
        const uint32_t up = (uint32_t)(seg >> 1) & 1u;
        if (!mbar_wait(&acce_bar[b], up ^ 1u, err)) {
          aborted = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dcol = tmem + (uint32_t)(b * ACC_COLS);
        const uint32_t idesc = pv.d->f16 ? IDESC_F16 : IDESC_BF16;
        uint32_t accum = 0;
        for (; w < wend; ++w, ++i) {
          const int s = (int)(i % stages);
          const uint32_t ph = (uint32_t)(i / stages) & 1u;
          const int bs = XQ ? (int)(i % bstages) : 0;
          const uint32_t bph = XQ ? (uint32_t)(i / bstages) & 1u : 0u;
          if (!mbar_wait(&full_bar[s], ph, err) || (XQ && !mbar_wait(&bfull_bar[bs], bph, err))) {
            aborted = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = saddr(smem + (size_t)s * ASTAGE);
          const uint32_t bh0 = a0 + A_BYTES;
          const uint32_t bl0 = bh0 + B_BYTES;
          if constexpr (XQ) {
            // factor slot bs: [hi K 0-63 | lo K 0-63 | hi K 64-127 | lo K
            // 64-127], each RP rows of 128 bytes, so the 2 RP rows of one
            // 64-wide K atom are contiguous 8-row groups (stride 1024 bytes)
#pragma unroll
            for (int kk = 0; kk < KB / 16; ++kk) {
              uint64_t da;
              if (MODE == 0) {
                const uint32_t aoff = (uint32_t)(kk / 4) * (A_BYTES / 2) + (uint32_t)(kk % 4) * 32;
                da = sdesc(a0 + aoff, 16, 1024);
              } else {
                da = sdesc(a0 + kk * 2048, A_BYTES / 2, 1024);
              }
              const uint32_t boff = (uint32_t)(kk / 4) * B_BYTES + (uint32_t)(kk % 4) * 32;
              mma_f16kind(dcol, da, sdesc(saddr(bring + (size_t)bs * BSLOT) + boff, 16, 1024),
                          IDESC_XQ, accum);
              accum = 1u;
            }
            mma_commit(&bempty_bar[bs]);   // factor slot free once these MMAs complete
          } else {
#pragma unroll
          for (int kk = 0; kk < KB / 16; ++kk) {
            uint64_t da, dbh, dbl;
            if (MODE == 0) {
              // K-major A and B: 16 elements = 32 bytes along the swizzled row;
              // K steps 4..7 live in the second 64-column box
              const uint32_t aoff = (uint32_t)(kk / 4) * BOXA + (uint32_t)(kk % 4) * 32;
              const uint32_t boff = (uint32_t)(kk / 4) * BOXB + (uint32_t)(kk % 4) * 32;
              da = sdesc(a0 + aoff, 16, 1024);
              dbh = sdesc(bh0 + boff, 16, 1024);
              dbl = sdesc(bl0 + boff, 16, 1024);
            } else {
              // MN-major A: 16 reduction rows = 2 x 1024 B; two 64-wide atoms
              // along the output index, 16 KB apart.  B: 64-element K atoms.
              da = sdesc(a0 + kk * 2048, A_BYTES / 2, 1024);
              const uint32_t boff = (uint32_t)(kk / 4) * BOXB + (uint32_t)(kk % 4) * 32;
              dbh = sdesc(bh0 + boff, 16, 1024);
              dbl = sdesc(bl0 + boff, 16, 1024);
            }
            mma_f16kind(dcol, da, dbh, idesc, accum);
            mma_f16kind(dcol, da, dbl, idesc, 1u);
            accum = 1u;
          }
          }
          mma_commit(&empty_bar[s]);
        }
        if (aborted) break;
        mma_commit(&accf_bar[b]);
      }
      mma_commit(&drain_bar);
    }
  } else if (XQ && warp >= 6) {
    // --------------------------------------------- FP8 -> BF16 converter
    // Warps 6..9.  Thread ct owns row ct of every tile: it reads the row's
    // 128 codes (eight 16-byte chunks, 128-byte swizzle: chunk c of row y
    // sits at position c ^ (y % 8)) and writes the row's 128 BF16 values
    // into the two 64-column boxes of the stage's A region with the same
    // swizzle, as a TMA copy of the BF16 tile would.  A quarter warp covers
    // eight consecutive rows, so both sides are free of bank conflicts.
    //
    // Codes are 0 or normal e4m3 (the staging flushes subnormal codes); for a
    // normal code c (exponent field e, mantissa m) the value c 2^k of a tile
    // with exponent k is 2^(e - 7 + k) (1 + m / 8), whose BF16 bits are
    // (c << 4) + ((120 + k) << 7): exponent e + 120 + k, mantissa m << 4.
    // Two codes are converted per 32-bit word as 16-bit lanes; the exponent
    // term is added only in lanes whose code is >= 8.
    griddep_wait();
    const int ct = threadIdx.x - 192;
    const int sw = ct & 7;
    int p = p0;
    ProbView<KB> pv;
    pv.load(probs, np, p, W);
    int64_t i = 0;
    // (every exit from this loop is warp-uniform: the warp meets __syncwarp
    // inside it)
    for (int64_t w = w0; w < w1; ++w, ++i) {
      if (__shfl_sync(0xffffffffu, *(volatile int*)&aborted, 0)) break;
      if (w >= pv.we) pv.load(probs, np, ++p, W);
      const int s = (int)(i % stages);
      const uint32_t ph = (uint32_t)(i / stages) & 1u;
      const int q = (int)(i % qstages);
      const uint32_t qph = (uint32_t)(i / qstages) & 1u;
      const int64_t lw = w - pv.wb;
      const int64_t tile = lw / pv.nkb, kb = lw % pv.nkb;
      // the tile's exponent: X tile (I, J) is (tile, kb) for X V and
      // (kb, tile) for X^T U (requested before the waits)
      const int64_t ti = MODE == 0 ? tile : kb, tj = MODE == 0 ? kb : tile;
      const uint32_t e0 = (uint32_t)(120 + __ldg(pv.d->xexp + ti * pv.d->ntj + tj));
      if (__any_sync(0xffffffffu, !mbar_wait(&qfull_bar[q], qph, err))) {
        aborted = 1;
        break;
      }
      // Convert into registers while the MMAs still read the A stage: only
      // the stores wait for it.
      const uint8_t* const src = qring + (size_t)q * Q_BYTES + ct * 128;
      uint4 in[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) in[c] = *reinterpret_cast<const uint4*>(src + ((c ^ sw) << 4));
      uint32_t o[64];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const uint32_t wv[4] = {in[c].x, in[c].y, in[c].z, in[c].w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t t = (wv[j] + 0x78787878u) & 0x80808080u;   // 0x80 where code >= 8
          o[8 * c + 2 * j] = __byte_perm(wv[j], 0, 0x4140) * 16u + __byte_perm(t, 0, 0x4140) * e0;
          o[8 * c + 2 * j + 1] =
              __byte_perm(wv[j], 0, 0x4342) * 16u + __byte_perm(t, 0, 0x4342) * e0;
        }
      }
      // every lane's codes are in registers: the FP8 slot can be refilled
      __syncwarp();
      if (lane == 0) mbar_arrive(&qempty_bar[q]);
      if (__any_sync(0xffffffffu, !mbar_wait(&empty_bar[s], ph ^ 1u, err))) {
        aborted = 1;
        break;
      }
      uint8_t* const sa = smem + (size_t)s * ASTAGE;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        // codes 16c..16c+15 = BF16 columns of box c / 4, chunks 2 (c % 4) and + 1
        uint8_t* const d = sa + (uint32_t)(c >> 2) * (A_BYTES / 2) + ct * 128;
        const int cc = (c & 3) * 2;
        *reinterpret_cast<uint4*>(d + ((cc ^ sw) << 4)) =
            make_uint4(o[8 * c], o[8 * c + 1], o[8 * c + 2], o[8 * c + 3]);
        *reinterpret_cast<uint4*>(d + (((cc + 1) ^ sw) << 4)) =
            make_uint4(o[8 * c + 4], o[8 * c + 5], o[8 * c + 6], o[8 * c + 7]);
      }
      // generic-proxy writes made visible to the tensor core's reads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&full_bar[s]);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // First the previous half step's deferred tail (HalfTail), if any, spread
    // over every CTA's four epilogue warps while the first accumulator fills.
    griddep_wait();   // the tail, out, corr, part and counters are shared
    {
      const HalfTail* tl = probs[0].tail;
      if (tl && __ldcg(&tl->pending))
        half_tail_work(tl, (int)blockIdx.x * 4 + (warp - 2), (int)gridDim.x * 4, lane);
    }
    // Warps 2..5: warp w reads TMEM lanes 32 (w % 4) .. + 31 (= tile rows).
    // The accumulator passes through a shared-memory tile with an odd row
    // stride (conflict-free), so that every global access below is a flat,
    // coalesced run: a 128-row tile of a dense rows x r array (out, corr, a
    // partial slot) is one contiguous block of 128 r floats.
    constexpr int SS = RP + 1;
    // (after the stage ring and, in the FP8 form, the FP8 tile ring)
    float* stg = reinterpret_cast<float*>(qring + (XQ ? (size_t)qstages * Q_BYTES : 0));
    const int quarter = warp & 3;
    const int lrow = quarter * 32 + lane;
    const int et = threadIdx.x - 64;                 // 0..127
    int p = p0;
    ProbView<KB> pv;
    pv.load(probs, np, p, W);
    int64_t seg = 0;
    for (int64_t w = w0; w < w1; ++seg) {
      if (w >= pv.we) pv.load(probs, np, ++p, W);
      const int r = pv.d->r;
      const int64_t rows_out = pv.d->rows_out;
      float* const out = pv.d->out;
      const float* const corr = pv.d->corr;
      const int q128 = 128 / r, r128 = 128 % r;      // a flat step of 128 as (rows, cols)
      const int rr0 = et / r, cc0 = et % r;
      const int64_t lw = w - pv.wb;
      const int64_t tile = lw / pv.nkb;
      const int64_t kb_a = lw % pv.nkb;
      const int64_t wend = min(w1, pv.wb + (tile + 1) * pv.nkb);
      const int64_t kb_b = wend - pv.wb - tile * pv.nkb;
      const int64_t nkb = pv.nkb;
      // the tile's first and one-past-last global units
      const int64_t gs = pv.wb + tile * nkb, ge = gs + nkb;
      w = wend;
      const int b = (int)(seg & 1);
      const uint32_t up = (uint32_t)(seg >> 1) & 1u;
      const bool whole = kb_a == 0 && kb_b == nkb;
      const int64_t row0 = tile * TILE;
      const int cnt = (int)min((int64_t)TILE, rows_out - row0) * r;
      // at rank <= 32 the corr values of a whole tile are requested before
      // its accumulator is ready (off the epilogue's critical path)
      constexpr int NPF = (RP <= 32 && !XQ) ? RP : 0;
      float cpre[NPF > 0 ? NPF : 1];
      if constexpr (NPF > 0) {
        if (whole && corr) {
          const float* cp = corr + row0 * r;
#pragma unroll
          for (int i = 0; i < NPF; ++i) {
            const int f = et + 128 * i;
            cpre[i] = f < cnt ? __ldcg(cp + f) : 0.f;
          }
        }
      }
      const bool ok = mbar_wait(&accf_bar[b], up, err);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // (no early exit on a failed wait: the four epilogue warps must all
      // reach the named barriers; the failed stores are skipped)
      asm volatile("bar.sync 1, 128;" ::: "memory");   // previous copy-out done
#pragma unroll
      for (int c0 = 0; c0 < RP; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * ACC_COLS + c0), v);
        if constexpr (XQ) {
          // X F_hi (columns 0..RP-1) + X F_lo (columns RP..2RP-1)
          float v2[16];
          tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * ACC_COLS + RP + c0), v2);
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] += v2[j];
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) stg[lrow * SS + c0 + j] = v[j];
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce_bar[b]);        // accumulator b free again
      asm volatile("bar.sync 1, 128;" ::: "memory");   // staging tile complete
      float* dst;
      const float* add = nullptr;
      if (whole) {
        dst = out + row0 * r;
        if (corr) add = corr + row0 * r;
      } else {
        const int slot = seg == 0 ? 0 : 1;
        dst = part + ((int64_t)blockIdx.x * 2 + slot) * TILE * RP;
      }
      if (ok) {
        int rr = rr0, cc = cc0;
        if constexpr (NPF > 0) {
#pragma unroll
          for (int i = 0; i < NPF; ++i) {
            const int f = et + 128 * i;
            if (f < cnt) {
              float v = stg[rr * SS + cc];
              if (add) v += cpre[i];
              dst[f] = v;
            }
            rr += q128;
            cc += r128;
            if (cc >= r) {
              cc -= r;
              ++rr;
            }
          }
        } else {
          // sixteen loads of the corr term in flight per thread, then their
          // stores (a load-add-store chain per element waits on one L2 round
          // trip at a time)
          constexpr int CHK = 16;
          for (int f0 = et; f0 < cnt; f0 += 128 * CHK) {
            float a[CHK];
#pragma unroll
            for (int u = 0; u < CHK; ++u) {
              const int f = f0 + 128 * u;
              a[u] = (add && f < cnt) ? __ldcg(add + f) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < CHK; ++u) {
              const int f = f0 + 128 * u;
              if (f < cnt) {
                float v = stg[rr * SS + cc];
                if (add) v += a[u];
                dst[f] = v;
                rr += q128;
                cc += r128;
                if (cc >= r) {
                  cc -= r;
                  ++rr;
                }
              }
            }
          }
        }
      }
      if (!whole && fixup) {
        // A tile cut by range boundaries: the last of its CTAs to get here
        // sums every contributor's slot, in CTA order (so the result does not
        // depend on which CTA is last), adds corr and writes the tile.
        // (Without fixup the slots are left for the consumer, which sums
        // them in the same order: tc_cut_row below.)
        __threadfence();
        asm volatile("bar.sync 1, 128;" ::: "memory");
        int64_t c_lo = blockIdx.x, c_hi = blockIdx.x;
        while (c_lo > 0 && sk_begin(c_lo, W, G) > gs) --c_lo;
        while (c_hi + 1 < G && sk_begin(c_hi + 1, W, G) < ge) ++c_hi;
        int* const cnt_t = &counters[pv.d->t_begin + tile];
        if (et == 0) {
          const int old = atomicAdd(cnt_t, 1);
          last_cta = old == (int)(c_hi - c_lo);
          if (last_cta) *cnt_t = 0;   // ready for the next launch
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (last_cta && ok) {
          __threadfence();
          // Per element: 0, plus each contributor's slot in CTA order, plus
          // corr.  float4 g of the flat tile goes to thread g % 128; the next
          // contributor's slot is loaded while the current one is added, so
          // the contributors' L2 round trips overlap.
          float* o = out + row0 * r;
          const float* cr = corr ? corr + row0 * r : nullptr;
          const bool vec = ((reinterpret_cast<uintptr_t>(o) | reinterpret_cast<uintptr_t>(cr)) & 15) == 0;
          const int n4 = vec ? cnt / 4 : 0;
          auto slot_of = [&](int64_t q) {
            const int slot = sk_begin(q, W, G) >= gs ? 0 : 1;
            return reinterpret_cast<const float4*>(part + (q * 2 + slot) * TILE * RP);
          };
          constexpr int CH = RP / 4 < 8 ? RP / 4 : 8;   // float4s per thread per chunk
          for (int g0 = 0; g0 * 128 < n4; g0 += CH) {
            float4 acc[CH], nxt[CH];
            const float4* src = slot_of(c_lo);
#pragma unroll
            for (int c = 0; c < CH; ++c) {
              const int g = et + 128 * (g0 + c);
              acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
              nxt[c] = g < n4 ? __ldcg(&src[g]) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            for (int64_t q = c_lo; q <= c_hi; ++q) {
              float4 cur[CH];
#pragma unroll
              for (int c = 0; c < CH; ++c) cur[c] = nxt[c];
              if (q < c_hi) {
                src = slot_of(q + 1);
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                  const int g = et + 128 * (g0 + c);
                  if (g < n4) nxt[c] = __ldcg(&src[g]);
                }
              }
#pragma unroll
              for (int c = 0; c < CH; ++c) {
                acc[c].x += cur[c].x;
                acc[c].y += cur[c].y;
                acc[c].z += cur[c].z;
                acc[c].w += cur[c].w;
              }
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
              const int g = et + 128 * (g0 + c);
              if (g < n4) {
                float4 v = acc[c];
                if (cr) {
                  const float4 a = reinterpret_cast<const float4*>(cr)[g];
                  v.x += a.x;
                  v.y += a.y;
                  v.z += a.z;
                  v.w += a.w;
                }
                reinterpret_cast<float4*>(o)[g] = v;
              }
            }
          }
          // elements past the last whole float4 (or all, when unaligned)
          for (int f = 4 * n4 + et; f < cnt; f += 128) {
            float sacc = 0.f;
            for (int64_t q = c_lo; q <= c_hi; ++q) {
              const int slot = sk_begin(q, W, G) >= gs ? 0 : 1;
              sacc += __ldcg(&part[(q * 2 + slot) * TILE * RP + f]);
            }
            o[f] = cr ? sacc + cr[f] : sacc;
          }
        }
      }
    }
  }
  __syncthreads();
  // every MMA the CTA issued has completed before tensor memory is freed
  mbar_wait(&drain_bar, 0, err);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// 16-bit conversions of the pairs (round to nearest even).
__device__ __forceinline__ __nv_bfloat16 to16(float v, __nv_bfloat16*) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ __half to16(float v, __half*) { return __float2half_rn(v); }
__device__ __forceinline__ float from16(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float from16(__half v) { return __half2float(v); }

// F (rows x r, FP32) -> F^T as a 16-bit pair (RP x ldt): hi = t(F),
// lo = t(F - hi), t the rounding to T.  Rows r..RP-1 of the outputs stay zero.
template <typename T>
__global__ void split_transpose_kernel(const float* __restrict__ F, int64_t rows, int r,
                                       T* __restrict__ hi, T* __restrict__ lo, int64_t ldt) {
  __shared__ float tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int64_t i = i0 + q;
    const int j = j0 + threadIdx.x;
    tile[q][threadIdx.x] = (i < rows && j < r) ? F[i * r + j] : 0.0f;
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int j = j0 + q;
    const int64_t i = i0 + threadIdx.x;
    if (j < r && i < rows) {
      const float v = tile[threadIdx.x][q];
      const T h = to16(v, (T*)nullptr);
      hi[(int64_t)j * ldt + i] = h;
      lo[(int64_t)j * ldt + i] = to16(v - from16(h), (T*)nullptr);
    }
  }
}

// X (FP32, m x n, ldx) -> X_hi = t(X), X_lo = t(X - X_hi), both m x ldh.
// ERR_DOMAIN for a negative or non-finite entry, or (FP16) one beyond the
// largest finite FP16 value.
template <typename T>
__global__ void split_x_kernel(const float* __restrict__ X, int64_t m, int64_t n, int64_t ldx,
                               T* __restrict__ xh, T* __restrict__ xl, int64_t ldh, float vmax,
                               int* err) {
  const int64_t total = m * n;
  int bad = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    const float v = X[i * ldx + j];
    if (!(v >= 0.0f) || isinf(v) || v > vmax) bad = 1;
    const T h = to16(v, (T*)nullptr);
    xh[i * ldh + j] = h;
    xl[i * ldh + j] = to16(v - from16(h), (T*)nullptr);
  }
  if (bad) atomicOr(err, ERR_DOMAIN);
}

// Exponent limits of the FP8 form's tile scales 2^k.  Below: tiles whose
// largest entry is under 448 * 2^-100 keep k = -100 (their entries become
// mostly zero codes and live in X_lo).  Above: X beyond 448 * 2^100 is
// outside the form (ERR_DOMAIN).  Both keep every BF16 exponent built by the
// converter (e + 120 + k, e in 1..15) inside the normal range.
constexpr int XQ_KMIN = -100, XQ_KMAX = 100;

// X (FP32, m x n, ldx) -> the FP8 stream form, one CTA per 128 x 128 tile
// (I, J) = (blockIdx.y, blockIdx.x):
//   k = min{k : amax <= 448 * 2^k} over the tile (exact, from frexp),
//       clamped below at XQ_KMIN;  xexp[I * ntj + J] = k;
//   q = e4m3_rn(x 2^-k) (x 2^-k <= 448, exact scaling); codes under 8
//       (zero and the subnormals, values below 2^-6) become 0; xq = q;
//   X_lo = bf16_rn(x - q 2^k) (the difference is exact in FP32).
// ERR_DOMAIN for a negative or non-finite entry, or amax > 448 * 2^XQ_KMAX.
__global__ void __launch_bounds__(256) quant_x_kernel(const float* __restrict__ X, int64_t m,
                                                      int64_t n, int64_t ldx,
                                                      uint8_t* __restrict__ xq, int64_t ldq,
                                                      __nv_bfloat16* __restrict__ xl, int64_t ldh,
                                                      int* __restrict__ xexp, int ntj, int* err) {
  __shared__ float wmax[8];
  __shared__ int kt;
  const int64_t i0 = (int64_t)blockIdx.y * 128, j0 = (int64_t)blockIdx.x * 128;
  const int rows = (int)min((int64_t)128, m - i0), cols = (int)min((int64_t)128, n - j0);
  float amax = 0.0f;
  int bad = 0;
  for (int e = threadIdx.x; e < 128 * 128; e += blockDim.x) {
    const int ii = e >> 7, jj = e & 127;
    if (ii < rows && jj < cols) {
      const float v = X[(i0 + ii) * ldx + j0 + jj];
      if (!(v >= 0.0f) || isinf(v)) bad = 1;
      else amax = fmaxf(amax, v);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = amax;
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = wmax[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) a = fmaxf(a, wmax[w]);
    int k = XQ_KMIN;
    if (a > 0.0f) {
      // a = f 2^e, f in [0.5, 1); 448 = 0.875 2^9
      int e;
      const float f = frexpf(a, &e);
      k = f <= 0.875f ? e - 9 : e - 8;
      if (k < XQ_KMIN) k = XQ_KMIN;
      if (k > XQ_KMAX) {
        k = XQ_KMAX;
        atomicOr(err, ERR_DOMAIN);
      }
    }
    kt = k;
    xexp[(int64_t)blockIdx.y * ntj + blockIdx.x] = k;
  }
  __syncthreads();
  const int k = kt;
  const float inv = __int_as_float((127 - k) << 23);   // 2^-k
  const float sc = __int_as_float((127 + k) << 23);    // 2^k
  for (int e = threadIdx.x; e < 128 * 128; e += blockDim.x) {
    const int ii = e >> 7, jj = e & 127;
    if (ii < rows && jj < cols) {
      const float v = X[(i0 + ii) * ldx + j0 + jj];
      uint8_t c = (uint8_t)(__nv_cvt_float_to_fp8(v * inv, __NV_SATFINITE, __NV_E4M3) & 0x7f);
      if (c < 8) c = 0;
      __half_raw hr = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)c, __NV_E4M3);
      const float hi = __half2float(__half(hr)) * sc;
      xq[(i0 + ii) * ldq + j0 + jj] = c;
      xl[(i0 + ii) * ldh + j0 + jj] = __float2bfloat16_rn(v - hi);
    }
  }
  if (bad) atomicOr(err, ERR_DOMAIN);
}

// Bounded-wait probe: one thread waits for something that never happens --
// kind 0: a global flag that nothing sets (the spin form of the grid
// barriers); kind 1: phase 0 of a shared-memory mbarrier that nothing arrives
// at (the form of the sweep's pipeline waits, through mbar_wait).  Both give
// up after `budget` cycles and record ERR_TIMEOUT in *err.
__global__ void probe_wait_kernel(int kind, long long budget, const unsigned int* flag, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  if (kind == 0) {
    const long long t0 = clock64();
    while (ld_acquire_gpu(flag) == 0u) {
      if (clock64() - t0 > budget) {
        atomicOr(err, ERR_TIMEOUT);
        break;
      }
    }
  } else {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait(&bar, 0u, err, budget);
  }
}

}  // namespace tc

// ------------------------------------------------------------------- host
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2D BF16 tensor map over a row-major (rows x cols, ld elements) array with a
// box of box_cols x box_rows and 128-byte swizzle.  Out-of-range reads give 0.
// f16: 0 = BF16, 1 = FP16, TC_MAP_U8 = one-byte codes (the FP8 form).
bool tc_make_map(void* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
                 int box_cols, int box_rows, int f16) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const int64_t es = f16 == TC_MAP_U8 ? 1 : 2;
  if (((uintptr_t)base & 15) || ((ld * es) & 15) || box_cols * es > 128) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = f16 == TC_MAP_U8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                 : f16            ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                  : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUresult r = fn(reinterpret_cast<CUtensorMap*>(map), dt, 2,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int tc_rank_pad(int r) { return r <= 16 ? 16 : (r <= 32 ? 32 : (r <= 48 ? 48 : 64)); }

// Dynamic shared memory: the stage ring (1024-byte aligned) and the
// epilogue's staging tile (TILE x (rp + 1) floats).
static size_t tc_staging(int rp) { return (size_t)tc::TILE * (rp + 1) * sizeof(float); }

static size_t tc_smem(int mode, int rp, int stages) {
  const int kb = mode == 0 ? tc::KB_XV : tc::KB_XT;
  return (size_t)stages * ((size_t)tc::TILE * kb * 2 + 2 * (size_t)rp * kb * 2) + 1024 +
         tc_staging(rp);
}

// FP8 form: two BF16 A stages (the converter fills one while the MMAs read
// the other), a ring of factor tiles (2 x rp x 128 BF16 pairs per unit; 3
// slots from rank pad 48 up, else 4) and as deep an FP8 tile ring as the
// rest of 227 KB allows (2 to 8 tiles): rank pad 64 -> 3 + 2, 48 -> 3 + 4,
// 32 -> 4 + 5, 16 -> 4 + 7.
static void tc_xq_plan(int mode, int rp, int* bstages, int* qstages, size_t* smem) {
  const int kb = mode == 0 ? tc::KB_XV : tc::KB_XT;
  const size_t a = (size_t)tc::TILE * kb * 2, bslot = 2 * (size_t)rp * kb * 2;
  const size_t budget = 227 * 1024 - 1024 - 1024 - tc_staging(rp) - 2 * a;
  const int nb = bslot >= 24576 ? 3 : 4;
  int q = (int)((budget - nb * bslot) / tc::Q_BYTES);
  q = q > 8 ? 8 : q;
  *bstages = nb;
  *qstages = q;
  *smem = 2 * a + nb * bslot + (size_t)q * tc::Q_BYTES + 1024 + tc_staging(rp);
}

// As many stages as fit in 227 KB per CTA (less 1 KB for static shared
// memory), between 2 and 8.
static int tc_stages(int mode, int rp) {
  const size_t budget = 227 * 1024 - 1024 - 1024 - tc_staging(rp);
  const int kb = mode == 0 ? tc::KB_XV : tc::KB_XT;
  const size_t st = (size_t)tc::TILE * kb * 2 + 2 * (size_t)rp * kb * 2;
  int s = (int)(budget / st);
  return s > 8 ? 8 : (s < 2 ? 2 : s);
}

// Grid of the persistent sweep: one CTA per SM, fewer when there are fewer
// k-blocks than SMs.
int tc_group_grid(int64_t W, int num_sms) {
  int64_t g = W < num_sms ? W : num_sms;
  if (g > tc::MAX_GRID) g = tc::MAX_GRID;
  return (int)(g < 1 ? 1 : g);
}

int tc_grid(int64_t rows_out, int64_t red, int mode, int num_sms) {
  const int kb = mode == 0 ? tc::KB_XV : tc::KB_XT;
  return tc_group_grid(((rows_out + tc::TILE - 1) / tc::TILE) * ((red + kb - 1) / kb), num_sms);
}

void tc_prob_sizes(int mode, SweepProb* d, int64_t rows_out, int64_t red, int r, int64_t w_begin,
                   int64_t t_begin, int64_t* units, int64_t* tiles) {
  const int kb = mode == 0 ? tc::KB_XV : tc::KB_XT;
  d->rows_out = rows_out;
  d->red = red;
  d->r = r;
  d->w_begin = w_begin;
  d->t_begin = t_begin;
  *tiles = (rows_out + tc::TILE - 1) / tc::TILE;
  *units = *tiles * ((red + kb - 1) / kb);
}

template <int MODE, int RP, bool XQ>
static void launch_tc(const SweepProb* probs, int np, int64_t W, float* part, int* counters,
                      int grid, int fixup, int* err, cudaStream_t s, int want_stages, int pdl) {
  const int max_st = tc_stages(MODE, RP);
  const int stages = XQ ? 2 : (want_stages >= 2 && want_stages < max_st ? want_stages : max_st);
  int qstages = 0, bstages = 0;
  size_t smem = tc_smem(MODE, RP, stages);
  if (XQ) tc_xq_plan(MODE, RP, &bstages, &qstages, &smem);
  cudaFuncSetAttribute(tc::sweep_tc_kernel<MODE, RP, XQ>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(XQ ? tc::THREADS_XQ : tc::THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, tc::sweep_tc_kernel<MODE, RP, XQ>, probs, np, W, stages, part, counters,
                     fixup, err, qstages, bstages);
}

void launch_tc_group(int mode, int rp, const SweepProb* probs, int np, int64_t W, float* part,
                     int* counters, int num_sms, int* err, cudaStream_t s, int fixup, int xq,
                     int stages, int pdl) {
  if (np < 1 || W < 1) return;
  const int grid = tc_group_grid(W, num_sms);
  note_launch(1);
#define TCL(M, P)                                                                       \
  (xq ? launch_tc<M, P, true>(probs, np, W, part, counters, grid, fixup, err, s, stages, pdl) \
      : launch_tc<M, P, false>(probs, np, W, part, counters, grid, fixup, err, s, stages, pdl))
  if (mode == 0) {
    if (rp == 16) TCL(0, 16); else if (rp == 32) TCL(0, 32); else if (rp == 48) TCL(0, 48); else TCL(0, 64);
  } else {
    if (rp == 16) TCL(1, 16); else if (rp == 32) TCL(1, 32); else if (rp == 48) TCL(1, 48); else TCL(1, 64);
  }
#undef TCL
}

void launch_split_transpose(const float* F, int64_t rows, int r, void* hi, void* lo, int64_t ldt,
                            int f16, cudaStream_t s) {
  note_launch(1);
  dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((r + 31) / 32));
  if (f16)
    tc::split_transpose_kernel<__half><<<grid, dim3(32, 8), 0, s>>>(F, rows, r, (__half*)hi,
                                                                    (__half*)lo, ldt);
  else
    tc::split_transpose_kernel<__nv_bfloat16><<<grid, dim3(32, 8), 0, s>>>(
        F, rows, r, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo, ldt);
}

void launch_split_x(const float* X, int64_t m, int64_t n, int64_t ldx, void* xh, void* xl,
                    int64_t ldh, int f16, int* err, cudaStream_t s) {
  note_launch(1);
  int64_t total = m * n;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 8192) blocks = 8192;
  if (f16)
    tc::split_x_kernel<__half><<<blocks, 256, 0, s>>>(X, m, n, ldx, (__half*)xh, (__half*)xl, ldh,
                                                      65504.0f, err);
  else
    tc::split_x_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(X, m, n, ldx, (__nv_bfloat16*)xh,
                                                             (__nv_bfloat16*)xl, ldh, INFINITY,
                                                             err);
}

void launch_quant_x(const float* X, int64_t m, int64_t n, int64_t ldx, void* xq, int64_t ldq,
                    void* xl, int64_t ldh, int* xexp, int* err, cudaStream_t s) {
  note_launch(1);
  const int ntj = (int)((n + 127) / 128);
  dim3 grid((unsigned)ntj, (unsigned)((m + 127) / 128));
  tc::quant_x_kernel<<<grid, 256, 0, s>>>(X, m, n, ldx, (uint8_t*)xq, ldq, (__nv_bfloat16*)xl,
                                          ldh, xexp, ntj, err);
}

}  // namespace enmf

using namespace enmf;

// Launches the bounded-wait probe and reports what its device status word says.
extern "C" enmf_status enmf_probe_wait(int32_t kind, int64_t cycles, int32_t* status) {
  if (!status || (kind != 0 && kind != 1) || cycles < 1 || cycles > 4000000000LL)
    return ENMF_EINVAL;
  void* buf = nullptr;
  if (cudaMalloc(&buf, 64) != cudaSuccess) {
    cudaGetLastError();
    return ENMF_ENOMEM;
  }
  int err = 0;
  cudaError_t e = cudaMemset(buf, 0, 64);
  if (e == cudaSuccess) {
    note_launch(1);
    tc::probe_wait_kernel<<<1, 32>>>(kind, cycles, (const unsigned int*)buf, (int*)buf + 4);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&err, (int*)buf + 4, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ENMF_ECUDA;
  }
  *status = (err & ERR_TIMEOUT) ? ENMF_ETIMEOUT : ENMF_OK;
  return ENMF_OK;
}
