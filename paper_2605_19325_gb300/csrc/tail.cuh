// The deferred tail of a HALS-stage half step (HalfTail, internal.h): run by
// the epilogue warps of the next tensor-core sweep pass while its first
// accumulator fills, or by the flush at the end of an enmf_iterate call.
// Every entry of the Gram is summed by one warp in the fixed order of
// warp_sum_partials, so the bits do not depend on which warp or launch runs
// it (and equal those of the half step's own reduction).
#pragma once

#include "internal.h"
#include "lanes.cuh"

namespace enmf {

// The end of the alternation (V-half): f = 1/2 ||X||^2 - <X^T U, V> +
// 1/2 <U^T U, V^T V> from the block partials, trace, counters, stage.
__device__ __forceinline__ void half_tail_finalize(const HalfTail* tl, int lane) {
  const int nb = tl->nb;
  double gg = 0.0, d = 0.0;
  for (int b = lane; b < nb; b += 32) {
    gg += __ldcg(&tl->obj_part[b]);
    if (tl->dot_part) d += __ldcg(&tl->dot_part[b]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gg += __shfl_xor_sync(lanes::FULL, gg, o);
    d += __shfl_xor_sync(lanes::FULL, d, o);
  }
  if (lane == 0) {
    DevState* st = tl->st;
    const volatile DevState* vs = st;
    const int stg = vs->stage, nu = vs->negU, nv = vs->negV;
    const double f = 0.5 * vs->normX2 - d + 0.5 * gg;
    st->f_last = f;
    if (tl->trace) tl->trace[tl->trace_idx] = f;
    if (stg == 0) st->asc_iters = vs->asc_iters + 1;
    else st->hals_iters = vs->hals_iters + 1;
    st->k = vs->k + 1;
    if (stg == 0 && !(nu || nv)) st->stage = 1;
    st->negU = 0;
    st->negV = 0;
  }
}

// Warp gw of ngw: its share of the Gram entries; warp 0 also the end of the
// alternation.
__device__ __forceinline__ void half_tail_work(const HalfTail* tl, int gw, int ngw, int lane) {
  const int kk = tl->kk, nb = tl->nb;
  for (int e = gw; e < kk; e += ngw) {
    const double s = lanes::warp_sum_partials(tl->gpart, nb, kk, e, lane);
    if (lane == 0) tl->G_out[e] = s;
  }
  if (gw == 0 && tl->finalize) half_tail_finalize(tl, lane);
}

}  // namespace enmf
