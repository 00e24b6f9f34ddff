// The ADMM rotation of Algorithm 1 for the forms with FP32 factors, every
// step of the loop inside one persistent cooperative kernel:
//   rows (all blocks)  for each row w of W = [U; V]: p = w R;
//                      y <- y + rho (z - p) from the second step on;
//                      b = p - y / rho;  z = prox(b) (Eq. 7);
//                      the block's share of M = W^T (z + y / rho);
//   M    (all blocks)  FP64 block partials, grid barrier, fixed-order sum;
//   R    (block 0)     R = polar(M), the orthogonal Procrustes solution
//                      (Sec. 4.1.2), by scaled Newton-Schulz in FP32 from
//                      M / ||M||_F until max |X^T X - I| < 1e-5 and one
//                      unscaled step more, then one step with X^T X - I summed
//                      in double-FP32: E is of the order of FP32 rounding, so
//                      R = X - X E / 2 needs X E only in FP32;
//   stop               ||R_new - R||_F <= tol sqrt(r), or max_iter steps.
// Rows use eight lanes per row with the entries in registers (lanes.cuh);
// nothing returns to the host between steps.
#include "internal.h"
#include "lanes.cuh"

namespace enmf {
namespace {

using namespace lanes;

constexpr int AT = 256;          // threads per block
constexpr int ARPB = AT / LPR;   // rows per block per pass

// Dynamic shared memory (floats): region A | X, X^T, P (KP x PLD each, rows
// padded by 4 floats: 16-byte aligned, and the rows that eight consecutive
// lanes read as float4 fall in distinct banks).  Region A holds Rs (KP^2) and
// ws, bs (32 KP each) in the row phase and the second X, X^T pair of the
// polar iteration on block 0.
template <int KP>
constexpr int polar_ld() { return KP + 4; }

template <int KP>
constexpr size_t admm_region_a() {
  const size_t rows = (size_t)KP * KP + 2 * (size_t)ARPB * KP;
  const size_t pol = 2 * (size_t)KP * polar_ld<KP>();
  return rows > pol ? rows : pol;
}

// ... followed, at KP <= 48, by the rows' w, z, y (ARPB x KP each) for when
// they stay resident (at KP = 64 that space would cost a block per SM).
template <int KP>
constexpr bool admm_resident_ok() { return KP <= 48; }

template <int KP>
constexpr size_t admm_smem() {
  return sizeof(float) * (admm_region_a<KP>() + 3 * (size_t)KP * polar_ld<KP>() +
                          (admm_resident_ok<KP>() ? 3 * (size_t)ARPB * KP : 0));
}

// acc[s1][s2] += sum_l A[ia_s1][l] B[jb_s2][l] over l < KP, with rows
// ia_s = bi + 16 s of A and jb_s = bj + 16 s of B (row stride LD), read as
// float4 along l.
template <int KP, int LD>
__device__ __forceinline__ void rows_dot(const float* __restrict__ A, const float* __restrict__ Bm,
                                         int bi, int bj, float (&acc)[KP / 16][KP / 16]) {
  constexpr int S = KP / 16;
#pragma unroll
  for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) acc[s1][s2] = 0.f;
  constexpr int UR = S <= 2 ? 4 : 1;
#pragma unroll UR
  for (int l = 0; l < KP; l += 4) {
    float4 x[S], y[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      x[s] = *reinterpret_cast<const float4*>(A + (bi + 16 * s) * LD + l);
      y[s] = *reinterpret_cast<const float4*>(Bm + (bj + 16 * s) * LD + l);
    }
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        float c = acc[s1][s2];
        c = fmaf(x[s1].x, y[s2].x, c);
        c = fmaf(x[s1].y, y[s2].y, c);
        c = fmaf(x[s1].z, y[s2].z, c);
        c = fmaf(x[s1].w, y[s2].w, c);
        acc[s1][s2] = c;
      }
  }
}

// Power iteration on I - P (P = X_0^T X_0, symmetric, eigenvalues in [0, 1])
// by warp 0, from the vector v of the previous call: the Rayleigh quotient mu
// gives sigma_min(X_0)^2 ~ 1 - mu (from above).  v: KP floats, zero past k.
template <int KP, int LD>
__device__ float sigma_min_estimate(const float* __restrict__ P, float* v, int k, int iters) {
  constexpr int E = (KP + 31) / 32;
  const int lane = threadIdx.x & 31;
  float w[E], mu = 0.f;
  for (int t = 0; t <= iters; ++t) {
#pragma unroll
    for (int e = 0; e < E; ++e) w[e] = lane + 32 * e < KP ? v[lane + 32 * e] : 0.f;
    for (int j = 0; j < k; ++j) {
      const float vj = v[j];
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (lane + 32 * e < KP) w[e] = fmaf(-P[j * LD + lane + 32 * e], vj, w[e]);
    }
    float nn = 0.f, vw = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (lane + 32 * e < KP) {
        nn = fmaf(w[e], w[e], nn);
        vw = fmaf(v[lane + 32 * e], w[e], vw);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nn += __shfl_xor_sync(FULL, nn, o);
      vw += __shfl_xor_sync(FULL, vw, o);
    }
    mu = vw;                                  // v is a unit vector
    if (t == iters || !(nn > 0.f)) break;
    const float inv = rsqrtf(nn);
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (lane + 32 * e < KP) v[lane + 32 * e] = w[e] * inv;
    __syncwarp();
  }
  return sqrtf(fmaxf(1.f - mu, 0.f));
}

// Two-sum of the running pair (hi, lo) and the exact product x y: hi + lo +
// x y = hi' + lo' up to the rounding of lo (the products are split by one
// FMA, the sum by Knuth's two-sum).  Explicit _rn operations: nothing may be
// contracted into an FMA.
__device__ __forceinline__ void dfloat_fma(float x, float y, float& hi, float& lo) {
  const float p = __fmul_rn(x, y);
  const float pe = fmaf(x, y, -p);
  const float sm = __fadd_rn(hi, p);
  const float bv = __fsub_rn(sm, hi);
  const float er = __fadd_rn(__fsub_rn(hi, __fsub_rn(sm, bv)), __fsub_rn(p, bv));
  hi = sm;
  lo = __fadd_rn(lo, __fadd_rn(er, pe));
}

__device__ __forceinline__ void dfloat_add(float& hi, float& lo, float h2, float l2) {
  const float sm = __fadd_rn(hi, h2);
  const float bv = __fsub_rn(sm, hi);
  const float er = __fadd_rn(__fsub_rn(hi, __fsub_rn(sm, bv)), __fsub_rn(h2, bv));
  hi = sm;
  lo = __fadd_rn(__fadd_rn(lo, l2), er);
}

// R = polar(M) on one block of AT threads (see the file comment).  X, XT and
// Y, YT: two KP x PLD buffer pairs (the iterate and the next one); P: KP x
// PLD; v: KP + 1 floats kept from step to step (the power-iteration vector
// and, in v[KP], the sigma_min estimate).  Thread (bi, bj) = (t / 16,
// t % 16) owns the entries (bi + 16 s1, bj + 16 s2).
//
// The iteration is Newton-Schulz with the scaling of a lower bound l of the
// singular values (X <- alpha X (3 I - alpha^2 X^T X) / 2, alpha^2 =
// 3 / (1 + l + l^2), which maps [l, 1] into [l', 1] with l' = alpha l (3 -
// alpha^2 l^2) / 2): for every singular value in (0, 1] it stays in (0, 1]
// and grows at least as fast as the unscaled step, so the limit is the same
// polar factor whatever l is; l only sets the speed.  l starts from a power
// iteration on I - X_0^T X_0.  The loop ends after the unscaled step that
// follows max |X^T X - I| < 1e-5 (the next step squares that deviation).
template <int KP>
__device__ void polar_block(const double* __restrict__ Mg, int k, double* R, double tol,
                            DevState* st, int* err, float* X, float* XT, float* Y, float* YT,
                            float* P, float* v, int step, double* sh) {
  const bool first = step == 0;
  constexpr int S = KP / 16, LD = polar_ld<KP>();
  constexpr int NM = (KP * KP + AT - 1) / AT;
  const int t = threadIdx.x, bi = t / 16, bj = t % 16;
  // M once (in FP32: any scale with sigma_max <= 1 serves)
  float mv[NM];
#pragma unroll
  for (int q = 0; q < NM; ++q) {
    const int e = t + AT * q, i = e / KP, j = e % KP;
    mv[q] = (e < KP * KP && i < k && j < k) ? (float)__ldcg(&Mg[i * k + j]) : 0.f;
  }
  float nl = 0.f;
#pragma unroll
  for (int q = 0; q < NM; ++q) nl = fmaf(mv[q], mv[q], nl);
  const float nf2 = block_sum256f(nl, reinterpret_cast<float*>(sh));
  const float inv = nf2 > 0.f ? 1.f / sqrtf(nf2) : 0.f;
#pragma unroll
  for (int q = 0; q < NM; ++q) {
    const int e = t + AT * q, i = e / KP, j = e % KP;
    if (e < KP * KP) {
      X[i * LD + j] = mv[q] * inv;
      XT[j * LD + i] = mv[q] * inv;
    }
  }
  if (first)
    for (int i = t; i < KP; i += AT) v[i] = i < k ? 1.f + 0.25f * (float)(i % 5) : 0.f;
  __syncthreads();
  float lk = 0.f;
  int it = 0;
  for (; it < 100; ++it) {
    float acc[S][S], xo[S][S];
    rows_dot<KP, LD>(XT, XT, bi, bj, acc);      // P = X^T X
    int ok = 1;
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        const int i = bi + 16 * s1, j = bj + 16 * s2;
        P[i * LD + j] = acc[s1][s2];
        xo[s1][s2] = X[i * LD + j];
        if (i < k && j < k && !(fabsf(acc[s1][s2] - (i == j ? 1.f : 0.f)) < 1e-5f)) ok = 0;
      }
    const bool conv = __syncthreads_and(ok) != 0;   // also orders P before its use
    if (it == 0) {
      // the estimate of sigma_min(X_0), refreshed every eighth step (M, and
      // with it the estimate, changes slowly from step to step) and kept in
      // v[KP] in between
      if (step % 8 == 0) {
        if (t < 32) {
          float l0 = sigma_min_estimate<KP, LD>(P, v, k, first ? 12 : 3);
          if (t == 0) v[KP] = fminf(fmaxf(0.9f * l0, 1e-4f), 1.f);
        }
        __syncthreads();
      }
      lk = v[KP];
    }
    const float al = conv ? 1.f : sqrtf(3.f / (1.f + lk + lk * lk));
    const float ca = 1.5f * al, cb = 0.5f * al * al * al;
    lk = 0.5f * al * lk * (3.f - al * al * lk * lk);
    rows_dot<KP, LD>(X, P, bi, bj, acc);        // X P  (P symmetric)
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        const int i = bi + 16 * s1, j = bj + 16 * s2;
        const float y = ca * xo[s1][s2] - cb * acc[s1][s2];
        Y[i * LD + j] = y;
        YT[j * LD + i] = y;
      }
    __syncthreads();
    float* tmp = X;
    X = Y;
    Y = tmp;
    tmp = XT;
    XT = YT;
    YT = tmp;
    if (conv) {
      ++it;
      break;
    }
  }
  // the old R, loaded while E is summed
  double rold[S][S];
#pragma unroll
  for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) {
      const int i = bi + 16 * s1, j = bj + 16 * s2;
      rold[s1][s2] = (i < k && j < k) ? __ldcg(&R[i * k + j]) : 0.0;
    }
  // E = X^T X - I to about 2^-44 (dfloat_fma, four chains over l mod 4; the
  // sub-blocks with bi <= bj, mirrored): E is of the order of FP32 rounding,
  // so R = X - X E / 2 needs X E only in FP32
  if (bi <= bj) {
#pragma unroll 1
    for (int c = 0; c < S * S; ++c) {
      const int i = bi + 16 * (c / S), j = bj + 16 * (c % S);
      const float* xi = XT + i * LD;
      const float* xj = XT + j * LD;
      float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f, h3 = 0.f, l3 = 0.f;
#pragma unroll 2
      for (int l = 0; l < KP; l += 4) {
        const float4 a4 = *reinterpret_cast<const float4*>(xi + l);
        const float4 b4 = *reinterpret_cast<const float4*>(xj + l);
        dfloat_fma(a4.x, b4.x, h0, l0);
        dfloat_fma(a4.y, b4.y, h1, l1);
        dfloat_fma(a4.z, b4.z, h2, l2);
        dfloat_fma(a4.w, b4.w, h3, l3);
      }
      dfloat_add(h0, l0, h1, l1);
      dfloat_add(h2, l2, h3, l3);
      dfloat_add(h0, l0, h2, l2);
      const float e = __fadd_rn(__fsub_rn(h0, (i == j && i < k) ? 1.f : 0.f), l0);
      P[i * LD + j] = e;
      P[j * LD + i] = e;
    }
  }
  __syncthreads();
  // R_new = X - X E / 2 (E symmetric), ||R_new - R||^2
  float acc[S][S];
  rows_dot<KP, LD>(X, P, bi, bj, acc);
  double d2 = 0.0;
#pragma unroll
  for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) {
      const int i = bi + 16 * s1, j = bj + 16 * s2;
      if (i < k && j < k) {
        const double rn = (double)X[i * LD + j] - 0.5 * (double)acc[s1][s2];
        const double x = rn - rold[s1][s2];
        d2 = fma(x, x, d2);
        R[i * k + j] = rn;
      }
    }
  d2 = block_sum256(d2, sh);
  if (t == 0) {
    const double dR = sqrt(d2);
    st->dR = dR;
    st->admm_steps = step + 1;   // (reset to 0 before the launch)
    st->jac_sweeps = it;
    if (!(nf2 > 0.f) || it >= 100) atomicOr(err, ERR_NOTCONV);
    if (dR <= tol * sqrt((double)k)) st->admm_done = 1;
  }
}

// The steps of one problem on its blocks lb = 0 .. nb - 1 (a whole grid, or
// a problem's share of a grouped grid); every grid barrier is `bar`, which
// all blocks of the grid pass.  GROUP: other problems share the grid, so a
// problem whose stop rule held keeps passing the barriers (without work)
// until max_iter instead of leaving the loop.
template <int KP, bool GROUP>
__device__ __forceinline__ void admm_body(const AdmmArgs& a, int lb, int nb, GridBarrier* bar,
                                          unsigned char* smraw, double* sh, float* pv) {
  constexpr int E = KP / LPR, S = KP / 16;
  float* Rs = reinterpret_cast<float*>(smraw);
  float* ws = Rs + KP * KP;
  float* bs = ws + ARPB * KP;
  float* X = Rs + admm_region_a<KP>();
  float* XT = X + KP * polar_ld<KP>();
  float* P = XT + KP * polar_ld<KP>();
  float* Y = Rs;                       // region A, polar only
  float* YT = Y + KP * polar_ld<KP>();
  float* wz = P + KP * polar_ld<KP>();  // resident rows: w | z | y, ARPB x KP each

  const int k = a.k, kk = k * k;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int sub = lane & (LPR - 1);
  const int rloc = warp * (32 / LPR) + lane / LPR;
  DevState* st = a.st;
  const int64_t m = a.m, rows = a.m + a.n;
  const int64_t passes = (rows + (int64_t)nb * ARPB - 1) / ((int64_t)nb * ARPB);
  const float rho = (float)a.rho;
  const float thr = -1.f / rho;

  // when every row fits in one pass a block owns the same rows at every step:
  // w, z and y then stay in shared memory from the first step to the last
  // (z and y are written back once, at the end); each thread touches only its
  // own entries there
  constexpr int NR = (KP * KP + AT - 1) / AT;
  const bool resident = admm_resident_ok<KP>() && passes == 1;
  float* wrow = wz + rloc * KP + sub;
  float* zrow = wrow + ARPB * KP;
  float* yrow = zrow + ARPB * KP;
  if (resident) {
    const int64_t i = (int64_t)lb * ARPB + rloc;
    const bool live = i < rows;
    float w[E], z[E], y[E];
    if (i < m) load_row(a.U, i, live, k, sub, w);
    else load_row(a.V, i - m, live, k, sub, w);
    load_row(a.Z, i, live, k, sub, z);
    load_row(a.Y, i, live, k, sub, y);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      wrow[LPR * e] = w[e];
      zrow[LPR * e] = z[e];
      yrow[LPR * e] = y[e];
    }
  }
  for (int step = 0; step < a.max_iter; ++step) {
    // the stop flag (the same value in every block) and R in one round trip
    const int done = *(volatile int*)&st->admm_done;
    float rv[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const int e = t + AT * q, i = e / KP, j = e % KP;
      rv[q] = (e < KP * KP && i < k && j < k) ? (float)__ldcg(&a.R[i * k + j]) : 0.f;
    }
    if (done) {
      if (!GROUP) break;
      // (the three barriers of the step, without its work)
      grid_sync(bar, a.err);
      grid_sync(bar, a.err);
      grid_sync(bar, a.err);
      continue;
    }
#pragma unroll
    for (int q = 0; q < NR; ++q)
      if (t + AT * q < KP * KP) Rs[t + AT * q] = rv[q];
    __syncthreads();
    float acc[S][S];
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) acc[s1][s2] = 0.f;
    for (int64_t ps = 0; ps < passes; ++ps) {
      const int64_t i = (ps * nb + lb) * ARPB + rloc;
      const bool live = i < rows;
      float w[E], z[E], y[E], p[E], bv[E];
      if (resident) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          w[e] = wrow[LPR * e];
          z[e] = zrow[LPR * e];
          y[e] = yrow[LPR * e];
        }
      } else {
        if (i < m) load_row(a.U, i, live, k, sub, w);
        else load_row(a.V, i - m, live, k, sub, w);
        load_row(a.Z, i, live, k, sub, z);
        load_row(a.Y, i, live, k, sub, y);
      }
      row_times<float, KP>(Rs, w, k, sub, p);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        float yy = y[e];
        if (step > 0) yy = yy + rho * (z[e] - p[e]);   // Y update of Algorithm 1
        const float b = p[e] - yy / rho;                // b = W R - Y / rho
        const float zz = b > 0.f ? b : (b >= thr ? 0.f : b + 1.f / rho);   // Eq. 7
        z[e] = zz;
        y[e] = yy;
        bv[e] = zz + yy / rho;                          // B = Z + Y / rho
      }
      if (resident) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          zrow[LPR * e] = z[e];
          yrow[LPR * e] = y[e];
        }
      } else {
        store_row(a.Z, i, live, k, sub, z);
        store_row(a.Y, i, live, k, sub, y);
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < E; ++e) {
        ws[rloc * KP + sub + LPR * e] = w[e];
        bs[rloc * KP + sub + LPR * e] = bv[e];
      }
      __syncthreads();
      accumulate_outer<float, KP>(ws, bs, ARPB, acc);
    }
    {
      const int bi = t / 16, bj = t % 16;
#pragma unroll
      for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) {
          const int pr = bi * S + s1, pc = bj * S + s2;
          if (pr < k && pc < k) a.part[(int64_t)lb * kk + pr * k + pc] = (double)acc[s1][s2];
        }
    }
    grid_sync(bar, a.err);
    sum_block_partials<AT>(a.part, nb, kk, a.M, 0, lb, nb);
    grid_sync(bar, a.err);
    if (lb == 0) polar_block<KP>(a.M, k, a.R, a.tol, st, a.err, X, XT, Y, YT, P, pv, step, sh);
    grid_sync(bar, a.err);
  }
  if (resident) {
    const int64_t i = (int64_t)lb * ARPB + rloc;
    float z[E], y[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      z[e] = zrow[LPR * e];
      y[e] = yrow[LPR * e];
    }
    store_row(a.Z, i, i < rows, k, sub, z);
    store_row(a.Y, i, i < rows, k, sub, y);
  }
}

template <int KP>
__global__ void __launch_bounds__(AT, KP <= 32 ? 3 : 2) admm_kernel(AdmmArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[AT];
  __shared__ float pv[KP + 1];
  admm_body<KP, false>(a, (int)blockIdx.x, (int)gridDim.x, &a.st->bar, smraw, sh, pv);
}

// Several problems of one rank pad in one cooperative grid: problem p owns
// blocks bbeg[p] .. bbeg[p + 1] - 1, as many as its own launch would have,
// so every problem's arithmetic (row partition, partial sums, polar) is that
// of its own launch; the barriers are `bar` for all.
template <int KP>
__global__ void __launch_bounds__(AT, KP <= 32 ? 3 : 2)
admm_group_kernel(const AdmmArgs* __restrict__ probs, const int* __restrict__ bbeg, int np,
                  GridBarrier* bar) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[AT];
  __shared__ float pv[KP + 1];
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
  __syncthreads();
  const int p = p_s;
  const AdmmArgs a = probs[p];
  admm_body<KP, true>(a, (int)blockIdx.x - bbeg[p], bbeg[p + 1] - bbeg[p], bar, smraw, sh, pv);
}

template <int KP>
int admm_capacity(int num_sms) {
  const size_t smem = admm_smem<KP>();
  cudaFuncSetAttribute(admm_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, admm_kernel<KP>, AT, smem);
  return (per < 1 ? 1 : per) * num_sms;
}

template <int KP>
void admm_launch(const AdmmArgs& a, int num_sms, cudaStream_t s) {
  const int64_t need = (a.m + a.n + ARPB - 1) / ARPB;
  int64_t grid = admm_capacity<KP>(num_sms);
  if (grid > NPART) grid = NPART;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  void* args[] = {(void*)&a};
  cudaLaunchCooperativeKernel((void*)admm_kernel<KP>, dim3((unsigned)grid), dim3(AT), args,
                              admm_smem<KP>(), s);
}

template <int KP>
int admm_group_capacity_k(int num_sms) {
  const size_t smem = admm_smem<KP>();
  cudaFuncSetAttribute(admm_group_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, admm_group_kernel<KP>, AT, smem);
  return (per < 1 ? 1 : per) * num_sms;
}

template <int KP>
void admm_group_launch(const AdmmArgs* probs, const int* bbeg, int np, int grid,
                       GridBarrier* bar, cudaStream_t s) {
  cudaFuncSetAttribute(admm_group_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)admm_smem<KP>());
  void* args[] = {(void*)&probs, (void*)&bbeg, (void*)&np, (void*)&bar};
  cudaLaunchCooperativeKernel((void*)admm_group_kernel<KP>, dim3((unsigned)grid), dim3(AT), args,
                              admm_smem<KP>(), s);
}

}  // namespace

int admm_group_capacity(int kp, int num_sms) {
  return kp == 16 ? admm_group_capacity_k<16>(num_sms) : kp == 32 ? admm_group_capacity_k<32>(num_sms)
         : kp == 48 ? admm_group_capacity_k<48>(num_sms) : admm_group_capacity_k<64>(num_sms);
}

int admm_blocks(int kp, int64_t rows, int num_sms) {
  const int64_t need = (rows + ARPB - 1) / ARPB;
  int64_t grid = kp == 16 ? admm_capacity<16>(num_sms) : kp == 32 ? admm_capacity<32>(num_sms)
                 : kp == 48 ? admm_capacity<48>(num_sms) : admm_capacity<64>(num_sms);
  if (grid > NPART) grid = NPART;
  if (grid > need) grid = need;
  return grid < 1 ? 1 : (int)grid;
}

void launch_admm_group(const AdmmArgs* probs, const int* bbeg, int np, int grid, int kp,
                       GridBarrier* bar, cudaStream_t s) {
  note_launch(1);
  if (kp == 16) admm_group_launch<16>(probs, bbeg, np, grid, bar, s);
  else if (kp == 32) admm_group_launch<32>(probs, bbeg, np, grid, bar, s);
  else if (kp == 48) admm_group_launch<48>(probs, bbeg, np, grid, bar, s);
  else admm_group_launch<64>(probs, bbeg, np, grid, bar, s);
}

void launch_admm_f32(const float* U, const float* V, int64_t m, int64_t n, int k, double* R,
                     float* Z, float* Y, double rho, int max_iter, double tol, DevState* st,
                     double* part, double* M, int* err, int num_sms, cudaStream_t s) {
  note_launch(1);
  AdmmArgs a{U, V, m, n, k, R, Z, Y, rho, max_iter, tol, st, part, M, err};
  const int kp = rank_pad16(k);
  if (kp == 16) admm_launch<16>(a, num_sms, s);
  else if (kp == 32) admm_launch<32>(a, num_sms, s);
  else if (kp == 48) admm_launch<48>(a, num_sms, s);
  else admm_launch<64>(a, num_sms, s);
}

}  // namespace enmf
