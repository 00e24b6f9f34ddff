// One half of an alternation of Algorithm 3: the rows of one factor F (U or
// V) updated with the other factor fixed.  Row i needs only its own row of F,
// its row of A (= X V or X^T U) and the r x r Gram G of the other factor
// (Sec. 4.2: the rows do not interact), so the rows run in parallel:
//   * HALS stage (Sec. 4.3): one sweep of the column updates
//       u_j <- max(0, u_j + (a_j - u . G_:j) / G_jj),  j = 1..r in order;
//   * ascent stage: the Eq. 8/9 shift of the negative entries, the mask of
//     Algorithm 2, and PBCD steps d_i = ||g_i||^2 / (g_i G g_i^T) (Eq. 10)
//     with the global stopping test of Algorithm 2 (a grid barrier);
// then the Gram F^T F of the updated factor, and at the end of the
// alternation (V-half) the objective f of Eq. 1 by the Gram expansion
//   f = 1/2 ||X||^2 - <X^T U, V> + 1/2 <U^T U, V^T V>
// and the stage decision, all inside one cooperative kernel.
//
// Mapping: eight lanes share a row; lane `sub` owns the entries
// l = sub + 8 e (e < KP / 8) of u, a and the gradient, in registers, for a
// rank padded to KP (16, 32, 48 or 64; padded entries are zero).  The HALS
// sweep keeps q = a - u G up to date: after u_j moves by delta the whole
// vector takes q <- q - delta G_j:, a rank-one update whose KP/8 FMAs per lane
// are independent, so a column step costs one shuffle and no dependent
// reduction chain.  Sums of a full row (u G, ||g||^2, g G g^T) combine the
// eight lanes by shuffles in a fixed pattern.
//
// The Gram of the block's rows is accumulated in TF by 16 x 16 threads, each
// owning a (KP/16) x (KP/16) sub-block, then written as an FP64 partial per
// block; after the grid barrier the partials are summed in block order.  The
// objective needs <U^T U, V^T V>, which is linear in the V^T V partials, so
// each block contributes <U^T U, its partial> and block 0 sums those scalars
// after the same barrier: one barrier per half step in the HALS stage.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "lanes.cuh"
#include "tail.cuh"

namespace enmf {
namespace {

using namespace lanes;

constexpr int HT = 256;          // threads per block
constexpr int RPB = HT / LPR;    // rows per block per pass

// Sum of n cross-block partials written before a grid barrier, by the whole
// block in a fixed order (L1 bypassed).  Every thread gets the result.
__device__ __forceinline__ double sum_partials(const double* p, int n, double* sh) {
  double s = 0.0;
  for (int b = threadIdx.x; b < n; b += HT) s += __ldcg(&p[b]);
  return block_sum256(s, sh);
}

// Adds the block's pass of rows (staged in `us`) to the thread's Gram
// sub-block.  Rows not present are zero.
template <typename TF, int KP>
__device__ __forceinline__ void gram_pass(TF* us, const TF (&u)[KP / LPR], int rloc, int sub,
                                          TF (&gacc)[KP / 16][KP / 16]) {
  constexpr int E = KP / LPR;
  __syncthreads();   // the previous pass has been consumed
#pragma unroll
  for (int e = 0; e < E; ++e) us[rloc * KP + sub + LPR * e] = u[e];
  __syncthreads();
  accumulate_outer<TF, KP>(us, us, RPB, gacc);
}

// The factor operand of the tensor-core sweeps: row i of F written to column
// i of th = t(F^T) and tl = t(F^T - th), t the rounding to BF16 or FP16 --
// the same rounding as the stand-alone split of tc_sweep.cu.  FP32 factors
// only.
template <typename TF, int E>
__device__ __forceinline__ void write_split(const HalfArgs& a, int64_t i, bool live, int k,
                                            int sub, const TF (&u)[E]) {
  if constexpr (sizeof(TF) == 4) {
    if (!a.th || !live) return;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int l = sub + LPR * e;
      if (l < k) {
        const int64_t o = (int64_t)l * a.ldt + i;
        if (a.t_f16) {
          const __half h = __float2half_rn(u[e]);
          reinterpret_cast<__half*>(a.th)[o] = h;
          reinterpret_cast<__half*>(a.tl)[o] = __float2half_rn(u[e] - __half2float(h));
        } else {
          const __nv_bfloat16 h = __float2bfloat16_rn(u[e]);
          reinterpret_cast<__nv_bfloat16*>(a.th)[o] = h;
          reinterpret_cast<__nv_bfloat16*>(a.tl)[o] = __float2bfloat16_rn(u[e] - __bfloat162float(h));
        }
      }
    }
  }
}

// Row i of A (X V or X^T U).  When the sweep left its cut tiles to the
// consumer (a.cut_part), a row of a cut tile is the sum of the contributing
// CTAs' slots in CTA order plus the X_lo term -- the order of the sweep's
// own fix-up, so the values are the same bits.  The contributors of the
// tile's units [gs, ge) under the stream-K split sk(c) = floor(c W / G) are
// c_lo = floor(((gs + 1) G - 1) / W) .. c_hi = floor((ge G - 1) / W).
template <typename TF, int E>
__device__ __forceinline__ void load_a_row(const HalfArgs& a, const TF* A, int64_t i, bool live,
                                           int k, int sub, TF (&v)[E]) {
  if constexpr (sizeof(TF) == 4) {
    if (a.sum_part) {
      // the fused kernel's per-cluster partials, summed in cluster order
      // (every load issued before the first add)
      float acc[E];
#pragma unroll
      for (int e = 0; e < E; ++e) acc[e] = 0.f;
      const int64_t stride = a.rows * (int64_t)k;
      const float* src = a.sum_part + i * k;
      int qq = 0;
      for (; qq + 4 <= a.sum_n; qq += 4) {
        float t[4][E];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int l = sub + LPR * e;
            t[u][e] = (live && l < k) ? __ldcg(src + (qq + u) * stride + l) : 0.f;
          }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int e = 0; e < E; ++e) acc[e] += t[u][e];
      }
      for (; qq < a.sum_n; ++qq)
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int l = sub + LPR * e;
          if (live && l < k) acc[e] += __ldcg(src + qq * stride + l);
        }
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int l = sub + LPR * e;
        v[e] = (live && l < k) ? (a.cut_corr ? acc[e] + a.cut_corr[i * k + l] : acc[e]) : TF(0);
      }
      return;
    }
    if (a.cut_part && live) {
      const int64_t W = a.cut_W, G = a.cut_G;
      const int64_t tile = i / 128;
      const int64_t gs = tile * a.cut_nkb, ge = gs + a.cut_nkb;
      const int64_t c_lo = ((gs + 1) * G - 1) / W, c_hi = (ge * G - 1) / W;
      if (c_lo != c_hi && c_hi - c_lo < 4) {
        // at most four contributors: every load issued before the first add
        float sl[4][E], cr[E];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          const int64_t q = c_lo + qq;
          const int slot = (q * W) / G >= gs ? 0 : 1;
          const float* src = a.cut_part + (q * 2 + slot) * 128 * a.cut_rp + (i % 128) * k;
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int l = sub + LPR * e;
            sl[qq][e] = (q <= c_hi && l < k) ? src[l] : 0.f;
          }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int l = sub + LPR * e;
          cr[e] = (a.cut_corr && l < k) ? a.cut_corr[i * k + l] : 0.f;
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int l = sub + LPR * e;
          float acc = 0.f;
#pragma unroll
          for (int qq = 0; qq < 4; ++qq)
            if (c_lo + qq <= c_hi) acc += sl[qq][e];
          v[e] = l < k ? (a.cut_corr ? acc + cr[e] : acc) : TF(0);
        }
        return;
      }
      if (c_lo != c_hi) {
        float acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.f;
        for (int64_t q = c_lo; q <= c_hi; ++q) {
          const int slot = (q * W) / G >= gs ? 0 : 1;
          const float* src = a.cut_part + (q * 2 + slot) * 128 * a.cut_rp + (i % 128) * k;
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int l = sub + LPR * e;
            if (l < k) acc[e] += src[l];
          }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int l = sub + LPR * e;
          v[e] = l < k ? (a.cut_corr ? acc[e] + a.cut_corr[i * k + l] : acc[e]) : TF(0);
        }
        return;
      }
    }
  }
  load_row(A, i, live, k, sub, v);
}

template <typename TF, int KP>
__device__ __forceinline__ void hstep_body(const HalfArgs& a, const int lb, const int nb,
                                           const int lock, TF* Gs, TF* us, TF* ginv,
                                           double* sh) {
  constexpr int E = KP / LPR, S = KP / 16;

  const int k = a.k;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int sub = lane & (LPR - 1);
  const int rloc = warp * (32 / LPR) + (lane / LPR);
  DevState* st = a.st;
  const int stage = *(volatile int*)&st->stage;
  TF* F = (TF*)a.F;
  const TF* A = (const TF*)a.A;
  const int64_t rows = a.rows;
  // the first pass's rows, requested before the Gram is staged so that the
  // two load latencies overlap
  const int64_t i_first = (int64_t)lb * RPB + rloc;
  TF u_first[E], a_first[E];
  load_row(F, i_first, i_first < rows, k, sub, u_first);
  if (!a.gram_only) load_a_row(a, A, i_first, i_first < rows, k, sub, a_first);
  if (a.G) {
#pragma unroll
    for (int q = 0; q < (KP * KP + HT - 1) / HT; ++q) {
      const int e = t + q * HT;
      if (e < KP * KP) {
        const int p = e / KP, c = e % KP;
        Gs[e] = (p < k && c < k) ? (TF)a.G[p * k + c] : TF(0);
      }
    }
  }
  __syncthreads();
  for (int j = t; j < KP; j += HT) {
    const TF g = Gs[j * KP + j];
    ginv[j] = g > TF(0) ? TF(1) / g : TF(0);
  }
  __syncthreads();

  const int64_t passes = (rows + (int64_t)nb * RPB - 1) / ((int64_t)nb * RPB);
  TF gacc[S][S];
#pragma unroll
  for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) gacc[s1][s2] = TF(0);
  double dotacc = 0.0;
  // the FP64 U^T U entries of this thread's Gram sub-block, for the objective
  // partial at the end (loaded now, off the critical path)
  double guv[S][S];
#pragma unroll
  for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) {
      const int p = (t / 16) * S + s1, c = (t % 16) * S + s2;
      guv[s1][s2] = (a.finalize && p < k && c < k) ? a.Gu[p * k + c] : 0.0;
    }

  if (a.gram_only) {
    for (int64_t ps = 0; ps < passes; ++ps) {
      const int64_t i = (ps * nb + lb) * RPB + rloc;
      TF u[E];
      if (ps == 0) {
#pragma unroll
        for (int e = 0; e < E; ++e) u[e] = u_first[e];
      } else {
        load_row(F, i, i < rows, k, sub, u);
      }
      write_split(a, i, i < rows, k, sub, u);
      gram_pass<TF, KP>(us, u, rloc, sub, gacc);
    }
  } else if (stage == 1) {
    // ---- HALS sweep over the columns, q = a - u G kept current
    for (int64_t ps = 0; ps < passes; ++ps) {
      const int64_t i = (ps * nb + lb) * RPB + rloc;
      const bool live = i < rows;
      TF u[E], av[E], q[E];
      if (ps == 0) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          u[e] = u_first[e];
          av[e] = a_first[e];
        }
      } else {
        load_row(F, i, live, k, sub, u);
        load_a_row(a, A, i, live, k, sub, av);
      }
      row_times<TF, KP>(Gs, u, k, sub, q);
#pragma unroll
      for (int e = 0; e < E; ++e) q[e] = av[e] - q[e];
      // column j's G row entries and 1 / G_jj are read one column ahead, off
      // the dependent chain (q_j -> u_j -> shuffle -> q update)
      TF gcol[E], gi = ginv[0];
#pragma unroll
      for (int ee = 0; ee < E; ++ee) gcol[ee] = Gs[sub + LPR * ee];
#pragma unroll
      for (int j = 0; j < KP; ++j) {
        if (j < k) {
          const int e = j / LPR, own = j % LPR;
          TF gnext[E], ginext = TF(0);
#pragma unroll
          for (int ee = 0; ee < E; ++ee) gnext[ee] = TF(0);
          if (j + 1 < KP) {
            ginext = ginv[j + 1];
#pragma unroll
            for (int ee = 0; ee < E; ++ee) gnext[ee] = Gs[(j + 1) * KP + sub + LPR * ee];
          }
          TF v = u[e], dl = TF(0);
          if (gi > TF(0)) {
            v = fma(q[e], gi, u[e]);
            v = v > TF(0) ? v : TF(0);
            dl = v - u[e];
          }
          dl = shfl8(dl, own);
          if (sub == own) u[e] = v;
#pragma unroll
          for (int ee = 0; ee < E; ++ee) q[ee] = fma(-dl, gcol[ee], q[ee]);
#pragma unroll
          for (int ee = 0; ee < E; ++ee) gcol[ee] = gnext[ee];
          gi = ginext;
        }
      }
      store_row(F, i, live, k, sub, u);
      write_split(a, i, live, k, sub, u);
      if (a.dot_part) {
#pragma unroll
        for (int e = 0; e < E; ++e) dotacc = fma((double)av[e], (double)u[e], dotacc);
      }
      gram_pass<TF, KP>(us, u, rloc, sub, gacc);
    }
  } else {
    // ---- ascent step: shift (Eq. 8/9), mask, PBCD (Algorithm 2)
    const TF sft = (TF)(a.which == 0 ? st->s_u : st->s_v);
    TF* gb = (TF*)a.gbuf;
    unsigned char* mk = reinterpret_cast<unsigned char*>(a.mask);
    double acc = 0.0;
    for (int64_t ps = 0; ps < passes; ++ps) {
      const int64_t i = (ps * nb + lb) * RPB + rloc;
      const bool live = i < rows;
      TF u[E], av[E], g[E];
      if (ps == 0) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          u[e] = u_first[e];
          av[e] = a_first[e];
        }
      } else {
        load_row(F, i, live, k, sub, u);
        load_a_row(a, A, i, live, k, sub, av);
      }
      unsigned bits = 0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        if (u[e] < TF(0)) u[e] = u[e] + sft;   // Eq. 8 / 9, literal (no clamp)
        if (u[e] >= TF(0)) bits |= 1u << e;
      }
      row_times<TF, KP>(Gs, u, k, sub, g);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        g[e] = ((bits >> e) & 1u) ? g[e] - av[e] : TF(0);
        acc = fma((double)g[e], (double)g[e], acc);
      }
      store_row(F, i, live, k, sub, u);
      store_row(gb, i, live, k, sub, g);
      if (live) mk[i * 8 + sub] = (unsigned char)bits;
    }
    double bsum = block_sum256(acc, sh);
    if (t == 0) a.part[lb] = bsum;
    grid_sync(a.bar, a.err);
    const double g0 = sqrt(sum_partials(a.part, nb, sh));
    int iters = 0;
    bool stopped = false;
    for (int it = 0; it < a.pbcd_max_iter; ++it) {
      acc = 0.0;
      for (int64_t ps = 0; ps < (stopped ? 0 : passes); ++ps) {
        const int64_t i = (ps * nb + lb) * RPB + rloc;
        const bool live = i < rows;
        TF u[E], av[E], g[E], tg[E];
        load_row(F, i, live, k, sub, u);
        load_row(gb, i, live, k, sub, g);
        load_a_row(a, A, i, live, k, sub, av);
        const unsigned bits = live ? mk[i * 8 + sub] : 0u;
        // d_i = ||g_i||^2 / (g_i G g_i^T)   (Eq. 10; App. B)
        row_times<TF, KP>(Gs, g, k, sub, tg);
        TF num = TF(0), den = TF(0);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          num = fma(g[e], g[e], num);
          den = fma(g[e], tg[e], den);
        }
        num = sum8(num);
        den = sum8(den);
        const TF d = (num > TF(0) && den > TF(0)) ? num / den : TF(0);
#pragma unroll
        for (int e = 0; e < E; ++e)
          if ((bits >> e) & 1u) {
            const TF v = u[e] - d * g[e];
            u[e] = v > TF(0) ? v : TF(0);   // (.)_+ of the PBCD update
          }
        row_times<TF, KP>(Gs, u, k, sub, g);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          g[e] = ((bits >> e) & 1u) ? g[e] - av[e] : TF(0);
          acc = fma((double)g[e], (double)g[e], acc);
        }
        store_row(F, i, live, k, sub, u);
        store_row(gb, i, live, k, sub, g);
      }
      double* pbuf = a.part + (size_t)((it + 1) & 1) * nb;
      bsum = block_sum256(acc, sh);
      if (t == 0) pbuf[lb] = bsum;
      grid_sync(a.bar, a.err);
      const double bc = sum_partials(pbuf, nb, sh);
      if (!stopped) {
        iters = it + 1;
        stopped = sqrt(bc) < a.eps * g0 || bc == 0.0;
      }
      if (stopped && lock < 0) break;
    }
    // entries still negative (unmasked) keep the ascent stage going
    int neg = 0;
    for (int64_t ps = 0; ps < passes; ++ps) {
      const int64_t i = (ps * nb + lb) * RPB + rloc;
      const bool live = i < rows;
      TF u[E];
      load_row(F, i, live, k, sub, u);
      write_split(a, i, live, k, sub, u);
      if (live) {
        const unsigned bits = mk[i * 8 + sub];
#pragma unroll
        for (int e = 0; e < E; ++e)
          if (sub + LPR * e < k && !((bits >> e) & 1u)) neg = 1;
        if (a.dot_part) {
          TF av[E];
          load_a_row(a, A, i, live, k, sub, av);
#pragma unroll
          for (int e = 0; e < E; ++e) dotacc = fma((double)av[e], (double)u[e], dotacc);
        }
      }
      gram_pass<TF, KP>(us, u, rloc, sub, gacc);
    }
    if (neg) atomicOr(a.which == 0 ? &st->negU : &st->negV, 1);
    if (lb == 0 && t == 0) {
      const int q = st->asc_iters;
      if (a.counts && 2 * q + a.which < a.counts_cap) a.counts[2 * q + a.which] = iters;
    }
  }

  if (lock > 0 && (a.gram_only || stage == 1)) {
    // keep pace with the ascending problems of the grid: the barriers of the
    // first PBCD pass and of every PBCD iteration
    for (int it = 0; it <= a.pbcd_max_iter; ++it) grid_sync(a.bar, a.err);
  }
  // ---- block partials: Gram (FP64), <A, F> and <U^T U, Gram partial>
  const int kk = k * k;
  {
    const int bi = t / 16, bj = t % 16;
    double obj = 0.0;
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        const int p = bi * S + s1, c = bj * S + s2;
        if (p < k && c < k) {
          const double gv = (double)gacc[s1][s2];
          a.gpart[(int64_t)lb * kk + p * k + c] = gv;
          if (a.finalize) obj = fma(guv[s1][s2], gv, obj);
        }
      }
    if (a.finalize) {
      obj = block_sum256(obj, sh);
      if (t == 0) a.obj_part[lb] = obj;
    }
  }
  if (a.dot_part) {
    const double dsum = block_sum256(dotacc, sh);
    if (t == 0) a.dot_part[lb] = dsum;
  }
  if (a.tail) {
    if (stage == 1 && !a.gram_only) {
      // HALS stage: the Gram sum and the end of the alternation are left to
      // the next sweep pass (no grid barrier here)
      if (lb == 0 && t == 0) {
        HalfTail* tl = a.tail;
        tl->gpart = a.gpart;
        tl->G_out = a.G_out;
        tl->obj_part = a.obj_part;
        tl->dot_part = a.dot_part;
        tl->st = a.st;
        tl->trace = a.trace;
        tl->nb = nb;
        tl->kk = kk;
        tl->finalize = a.finalize;
        tl->trace_idx = a.trace_idx;
        tl->pending = 1;
      }
      return;
    }
    if (lb == 0 && t == 0) a.tail->pending = 0;
  }
  grid_sync(a.bar, a.err);

  // ---- G_out = sum of the block partials in block order (block 0 left free
  // for the end-of-alternation work when there are other blocks)
  sum_block_partials<HT>(a.gpart, nb, kk, a.G_out, (a.finalize && nb > 1) ? 1 : 0, lb, nb);
  if (!a.finalize || lb != 0) return;

  // ---- end of the alternation (block 0): objective and stage update.  The
  // state is read in one go (its loads overlap the partial sums) and both
  // sums share one block reduction (each in the order of sum_partials).
  int stg = 0, nu = 0, nv = 0, asc = 0, hal = 0, kk0 = 0;
  double nx2 = 0.0;
  if (t == 0) {
    const volatile DevState* vs = st;
    stg = vs->stage;
    nu = vs->negU;
    nv = vs->negV;
    asc = vs->asc_iters;
    hal = vs->hals_iters;
    kk0 = vs->k;
    nx2 = vs->normX2;
  }
  double gg = 0.0, d = 0.0;
  for (int b = t; b < nb; b += HT) {
    gg += __ldcg(&a.obj_part[b]);
    d += __ldcg(&a.dot_part[b]);
  }
  block_sum256x2(gg, d, sh);
  if (t == 0) {
    const double f = 0.5 * nx2 - d + 0.5 * gg;
    st->f_last = f;
    if (a.trace) a.trace[a.trace_idx] = f;
    if (stg == 0) st->asc_iters = asc + 1;
    else st->hals_iters = hal + 1;
    st->k = kk0 + 1;
    if (stg == 0 && !(nu || nv)) st->stage = 1;
    st->negU = 0;
    st->negV = 0;
  }
}

template <typename TF, int KP>
__global__ void __launch_bounds__(HT) hstep_kernel(HalfArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TF* Gs = reinterpret_cast<TF*>(smraw);   // KP x KP, zero padded
  TF* us = Gs + KP * KP;                   // RPB x KP rows of the current pass
  __shared__ double sh[HT];
  __shared__ TF ginv[KP];                  // 1 / G_jj (0 where G_jj <= 0)
  // (a programmatic dependent of the sweep it reads: nothing before the wait;
  // then the next sweep may start requesting its X tiles)
  griddep_wait();
  griddep_launch();
  hstep_body<TF, KP>(a, (int)blockIdx.x, (int)gridDim.x, -1, Gs, us, ginv, sh);
}

// Grouped half steps: problem p (descriptors in device memory) owns blocks
// bbeg[p] .. bbeg[p + 1] - 1 of the grid; every descriptor's `bar` is the
// same grid barrier.
template <typename TF, int KP>
__global__ void __launch_bounds__(HT) hstep_group_kernel(const HalfArgs* __restrict__ probs,
                                                         const int* __restrict__ bbeg, int np) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TF* Gs = reinterpret_cast<TF*>(smraw);
  TF* us = Gs + KP * KP;
  __shared__ double sh[HT];
  __shared__ TF ginv[KP];
  __shared__ int p_s;
  if (threadIdx.x == 0) {
    int lo = 0, hi = np - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (bbeg[mid] <= (int)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    p_s = lo;
  }
  // some problem of the grid in the ascent stage (read before any barrier,
  // so every block sees the same stages)
  int asc = 0;
  for (int q = threadIdx.x; q < np; q += HT)
    if (!probs[q].gram_only && *(volatile int*)&probs[q].st->stage == 0) asc = 1;
  const int lock = __syncthreads_or(asc) ? 1 : 0;
  const int p = p_s;
  hstep_body<TF, KP>(probs[p], (int)blockIdx.x - bbeg[p], bbeg[p + 1] - bbeg[p], lock, Gs, us,
                     ginv, sh);
}

// The pending tails of a call's last half steps (one block of four warps).
// The flush spreads each pending tail's Gram entries over every warp of the
// grid; the pending flags are cleared by a second launch, once all of them are
// done.
__global__ void __launch_bounds__(128) half_tail_flush_kernel(const HalfTail* tails, int n) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * 4 + (threadIdx.x >> 5), ngw = gridDim.x * 4;
  for (int i = 0; i < n; ++i)
    if (__ldcg(&tails[i].pending)) half_tail_work(tails + i, gw, ngw, lane);
}

__global__ void half_tail_clear_kernel(HalfTail* tails, int n) {
  if (threadIdx.x < n) tails[threadIdx.x].pending = 0;
}

template <typename TF, int KP>
size_t hstep_smem() {
  return sizeof(TF) * ((size_t)KP * KP + (size_t)RPB * KP);
}

template <typename TF, int KP>
int hstep_capacity(int num_sms) {
  const size_t smem = hstep_smem<TF, KP>();
  cudaFuncSetAttribute(hstep_kernel<TF, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, hstep_kernel<TF, KP>, HT, smem);
  return (per < 1 ? 1 : per) * num_sms;
}

template <typename TF, int KP>
void hstep_launch(const HalfArgs& a, int grid, cudaStream_t s, int pdl) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(HT);
  cfg.dynamicSmemBytes = hstep_smem<TF, KP>();
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 2 : 1;
  cudaLaunchKernelEx(&cfg, hstep_kernel<TF, KP>, a);
}

}  // namespace

// Largest co-resident grid of the half step for this form and rank, at most
// NPART blocks (the size of the partial buffers).
int half_step_grid(int fdt, int k, int num_sms, int64_t rows) {
  const int kp = rank_pad16(k);
  int cap;
  if (fdt == T_F64)
    cap = kp == 16 ? hstep_capacity<double, 16>(num_sms) : kp == 32 ? hstep_capacity<double, 32>(num_sms)
          : kp == 48 ? hstep_capacity<double, 48>(num_sms) : hstep_capacity<double, 64>(num_sms);
  else
    cap = kp == 16 ? hstep_capacity<float, 16>(num_sms) : kp == 32 ? hstep_capacity<float, 32>(num_sms)
          : kp == 48 ? hstep_capacity<float, 48>(num_sms) : hstep_capacity<float, 64>(num_sms);
  if (cap > NPART) cap = NPART;
  // no more blocks than the rows fill in one pass
  const int64_t need = (rows + RPB - 1) / RPB;
  return need < 1 ? 1 : (need < cap ? (int)need : cap);
}

template <int K>
static int group_capacity(int num_sms) {
  const size_t smem = hstep_smem<float, K>();
  cudaFuncSetAttribute(hstep_group_kernel<float, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, hstep_group_kernel<float, K>, HT, smem);
  return (per < 1 ? 1 : per) * num_sms;
}

int half_group_capacity(int kp, int num_sms) {
  return kp == 16 ? group_capacity<16>(num_sms)
         : kp == 32 ? group_capacity<32>(num_sms)
         : kp == 48 ? group_capacity<48>(num_sms)
                    : group_capacity<64>(num_sms);
}

void launch_half_group(const HalfArgs* probs, const int* bbeg, int np, int grid, int kp,
                       cudaStream_t s) {
  note_launch(1);
  void* args[] = {(void*)&probs, (void*)&bbeg, (void*)&np};
#define HGL(K)                                                                                  \
  cudaLaunchCooperativeKernel((void*)hstep_group_kernel<float, K>, dim3(grid), dim3(HT), args, \
                              hstep_smem<float, K>(), s)
  if (kp == 16) HGL(16);
  else if (kp == 32) HGL(32);
  else if (kp == 48) HGL(48);
  else HGL(64);
#undef HGL
}

void launch_half_tail_flush(HalfTail* tails, int n, int num_sms, cudaStream_t s) {
  note_launch(2);
  half_tail_flush_kernel<<<num_sms, 128, 0, s>>>(tails, n);
  half_tail_clear_kernel<<<1, 32, 0, s>>>(tails, n);
}

void launch_half_step(const HalfArgs& a, int grid, cudaStream_t s, int pdl) {
  note_launch(1);
  const int64_t need = (a.rows + RPB - 1) / RPB;
  if ((int64_t)grid > need) grid = (int)need;
  if (grid < 1) grid = 1;
  const int kp = rank_pad16(a.k);
  if (a.fdt == T_F64) {
    if (kp == 16) hstep_launch<double, 16>(a, grid, s, pdl);
    else if (kp == 32) hstep_launch<double, 32>(a, grid, s, pdl);
    else if (kp == 48) hstep_launch<double, 48>(a, grid, s, pdl);
    else hstep_launch<double, 64>(a, grid, s, pdl);
  } else {
    if (kp == 16) hstep_launch<float, 16>(a, grid, s, pdl);
    else if (kp == 32) hstep_launch<float, 32>(a, grid, s, pdl);
    else if (kp == 48) hstep_launch<float, 48>(a, grid, s, pdl);
    else hstep_launch<float, 64>(a, grid, s, pdl);
  }
}

}  // namespace enmf
