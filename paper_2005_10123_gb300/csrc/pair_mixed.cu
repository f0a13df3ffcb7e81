// Mixed-precision pair kernel: float32 pair terms, float32 accumulation over one
// kColTile-column tile, float64 accumulation across tiles and items.
//
// For every row (event n) of its row tile the kernel forms, over the columns n' of its
// work range (Section 2.1, Eq. 1 inner sum; the gradient moments are added here):
//   S_b = sum_n'           e_b,   e_b = exp(-r^2/(2 tau_x^2) - dt^2/(2 tau_t^2))
//   S_s = sum_{t_n' < t_n} e_s,   e_s = exp(-omega dt - r^2/(2 h^2))
//   R_b = sum r^2 e_b,  T_b = sum dt'^2 e_b,  R_s = sum r^2 e_s,  U_s = sum dt e_s
// with r^2 = |x_n - x_n'|^2 and, for the background, dt' = beta (t_n - t_n'), beta^2 =
// log2(e)/(2 tau_t^2): times enter relative to the first row of the tile before scaling, and
// each scaled time (and scaled coordinate) is the correctly rounded product with the float64
// scale (scale_split), so no float32 rounding of a bandwidth biases the sums. The trigger
// terms take dt = t_n - t_n' from the stored float32 times (one rounding), so a trigger that
// decays within a small part of the tile's time span keeps full relative precision. The CTA
// that completes a row tile's merge tree turns its row sums into lambda_n, log lambda_n and
// the gradient in float64 (fused epilogue).
//
// Arithmetic per (row, column) pair, two rows per packed f32x2 value:
//   e_b = 2^-q with q = a2 r^2 + dt'^2, a2 = s^2 = log2(e)/(2 tau_x^2);
//   e_s = 2^(cn r^2 + w dt), cn = -log2(e)/(2 h^2), w = -omega log2(e).
// Tiles with background terms only (most of the window) take the differences of coordinates
// pre-scaled by s, q = (s dx)^2 + (s dy)^2 + dt'^2; tiles with trigger terms take r^2 from
// exact float32 differences of the stored coordinates. Sum 2 accumulates Q = sum q e_b, and
// the epilogue forms R_b = (Q - T_b) / s^2 in float64.
// In tiles where every pair is causal the trigger factor 2^(w dt) splits into a column
// factor 2^(w (t_ref - t_n')) folded into the exponent and a row factor 2^(w (t_n - t_ref))
// applied to the tile's trigger sums, with t_ref the tile's latest column time (both factors
// <= 1).
// The causal indicator t_n' < t_n is tested on stored times through lo[n] (the first
// index whose stored time equals t_n): for sorted times, t_n' < t_n  <=>  n' < lo[n].
// Column tiles entirely before a warp's rows skip the test, tiles entirely after skip the
// trigger term; only tiles straddling the rows test pair by pair.
//
// The HK_PACK_* switches choose, per operation kind, packed f32x2 instructions or two
// scalar ones (same rounding either way: each is one IEEE round-to-nearest operation).
#include <type_traits>

#include "hk_internal.h"

#ifndef HK_MIN_CTAS
#define HK_MIN_CTAS 10  // resident CTAs per SM, loglik + gradient (shared memory allows 10)
#endif
#ifndef HK_MIN_CTAS_LL
#define HK_MIN_CTAS_LL 12  // resident CTAs per SM, loglik only (80 registers, no spills)
#endif
#ifndef HK_MIN_CTAS_MIX
#define HK_MIN_CTAS_MIX 7  // resident CTAs per SM, two-component trigger mixture, loglik + gradient (shared memory allows 7)
#endif
#ifndef HK_MIN_CTAS_MIX_LL
#define HK_MIN_CTAS_MIX_LL 8  // two-component trigger mixture, loglik only
#endif
#ifndef HK_COL_UNROLL
#define HK_COL_UNROLL 8  // columns unrolled per step of the tile loop, loglik + gradient
#endif
#ifndef HK_COL_UNROLL_SEP
#define HK_COL_UNROLL_SEP 4  // separable trigger tiles, loglik + gradient (8 spills registers)
#endif
#ifndef HK_COL_UNROLL_LL
#define HK_COL_UNROLL_LL 8  // loglik only
#endif
#ifndef HK_SYM_UNROLL
#define HK_SYM_UNROLL 1  // steps unrolled in the far (shared-background) tile pass, loglik + gradient
#endif
#ifndef HK_SYM_UNROLL_LL
#define HK_SYM_UNROLL_LL 3  // the same, loglik only
#endif
#ifndef HK_NEAR_UNROLL
#define HK_NEAR_UNROLL 2  // steps unrolled in the shared near tile pass, loglik + gradient
#endif
#ifndef HK_NEAR_UNROLL_LL
#define HK_NEAR_UNROLL_LL HK_NEAR_UNROLL  // the same, loglik only
#endif
#ifndef HK_SNEAR_WEIGHT
#define HK_SNEAR_WEIGHT 19  // cost of a shared near column tile in tenths of a row-by-row one
#endif
#ifndef HK_FAR_WEIGHT
#define HK_FAR_WEIGHT 10  // cost of a far column tile in tenths of a near one, for the leaf split
#endif
#ifndef HK_PACK_ADD
#define HK_PACK_ADD 1  // differences dx, dy, dt
#endif
#ifndef HK_PACK_MUL
#define HK_PACK_MUL 1
#endif
#ifndef HK_PACK_FMA
#define HK_PACK_FMA 1
#endif
#ifndef HK_PACK_ACC
#define HK_PACK_ACC 1  // accumulation of the exponentials
#endif

namespace hk {
namespace {

constexpr double kLog2eD = 1.4426950408889634074;  // log2(e)
constexpr float kPadScaled = 1.0e18f;  // scaled time of a padded event: dt'^2 = 1e36 stays finite

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) {
#if HK_PACK_ADD
  return __fadd2_rn(a, b);
#else
  return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y));
#endif
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
#if HK_PACK_MUL
  return __fmul2_rn(a, b);
#else
  return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y));
#endif
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
#if HK_PACK_FMA
  return __ffma2_rn(a, b, c);
#else
  return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
#endif
}
__device__ __forceinline__ float2 acc2(float2 s, float2 e) {
#if HK_PACK_ACC
  return __fadd2_rn(s, e);
#else
  return make_float2(__fadd_rn(s.x, e.x), __fadd_rn(s.y, e.y));
#endif
}
__device__ __forceinline__ float2 accfma2(float2 a, float2 e, float2 s) {
#if HK_PACK_ACC
  return __ffma2_rn(a, e, s);
#else
  return make_float2(__fmaf_rn(a.x, e.x, s.x), __fmaf_rn(a.y, e.y, s.y));
#endif
}

constexpr int kPairs = kRowsPerThread / 2;  // packed row pairs per thread
constexpr int kColUnroll = HK_COL_UNROLL, kColUnrollLL = HK_COL_UNROLL_LL;
constexpr int kColUnrollSep = HK_COL_UNROLL_SEP;

template <int NS>
struct Acc32 {
  float2 v[NS][kPairs];
};

// One column tile against this thread's rows. KIND 0: background only (no causal pair, or
// every trigger term of the tile is exactly zero); 1: every pair causal (separable trigger
// factor); 2: test each pair (and mask n' = n when excluding self); 3: every pair causal and
// every background term exactly zero (trigger only, separable).
// KIND 0 reads the scaled coordinates (X, Y and sxs hold s x, s y with s^2 = a2), so that
// q = (s dx)^2 + (s dy)^2 + dt'^2 takes two FMAs after dt'^2. The other kinds read the stored
// coordinates, because the trigger term's Gaussian is narrow (h) and needs r^2 from exact
// differences: there q = a2 r^2 + dt'^2 with a2 = s*s rounded. Every kind accumulates the
// background moment Q = sum q e_b in sum 2; the epilogue recovers R_b = (Q - T_b) / s^2.
// The trigger terms take their time differences from the stored (unscaled, unshifted) float32
// times, dt = t_n - t_n' rounded once (exact where t_n' >= t_n / 2), with the slope WN = -omega
// log2(e) per unit of time: the background's scaled times t' = beta (t - t_origin) carry an
// absolute rounding error of about 2^-24 |t'|, which a trigger decaying within a small part of
// the row tile's time span (omega times the span large) would feel as a relative error of
// omega 2^-24 |t - t_origin| in each term. The moment U_s = sum dt e_s is therefore in units of
// time (rowtile_epilogue converts it). The separable column factor b = WN (t_ref - t') is formed
// per column from the staged stored time: one rounded difference, then one rounded product.
// With a two-component trigger mixture (MIX = 2) the trigger terms are formed for the components
// in COMP (bit 0: component 1, bit 1: component 2 with CN2, WN2, into the sums after the
// single-kernel ones); the caller leaves out a component whose terms are all exactly zero.
template <int KIND, bool GRAD, int MIX, int COMP = 1>
__device__ __forceinline__ void tile_pass(const float4 *__restrict__ sxs, const float4 *__restrict__ stx,
                                          const float *__restrict__ srt, const float2 (&X)[kPairs],
                                          const float2 (&Y)[kPairs], const float2 (&T)[kPairs],
                                          const float2 (&TR)[kPairs], const int (&LO)[kRowsPerThread],
                                          int row_a0, int c0, bool excl, float2 A2, float2 CN, float2 WN,
                                          float2 CN2, float2 WN2, float2 SREF,
                                          Acc32<num_sums(GRAD, MIX)> &acc) {
  constexpr int S2 = GRAD ? 6 : 2;  // component 2's trigger sum (then R_s2, U_s2 with the gradient)
  constexpr bool kC1 = (COMP & 1) != 0, kC2 = MIX > 1 && (COMP & 2) != 0;
  constexpr bool kBg = KIND != 3;
  constexpr bool kTrig = KIND != 0;
  constexpr bool kNeedDt = kBg;                               // scaled dt' (background)
  constexpr bool kNeedDtr = KIND == 2;                        // stored-time dt (trigger, per pair)
  constexpr int kUnroll = GRAD ? ((KIND == 1 || KIND == 3) ? kColUnrollSep : kColUnroll) : kColUnrollLL;
  if constexpr (KIND == 0 && !GRAD) {
    // background only, loglik: the unused trigger sum holds the odd columns' background sum,
    // halving the dependent chain of the accumulation (1.4% faster loglik; no gain with the
    // gradient, whose three chains already interleave)
#pragma unroll kUnroll / 2
    for (int j = 0; j < kColTile; j += 2) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4 d = stx[j + h], c = sxs[j + h];
        const float2 ct = make_float2(d.x, d.y), cx = make_float2(c.x, c.y), cy = make_float2(c.z, c.w);
#pragma unroll
        for (int p = 0; p < kPairs; ++p) {
          const float2 dx = add2(X[p], cx), dy = add2(Y[p], cy), dt = add2(T[p], ct);
          const float2 q = fma2(dy, dy, fma2(dx, dx, mul2(dt, dt)));
          acc.v[h][p] = acc2(acc.v[h][p], make_float2(ex2(-q.x), ex2(-q.y)));
        }
      }
    }
#pragma unroll
    for (int p = 0; p < kPairs; ++p) {
      acc.v[0][p] = acc2(acc.v[0][p], acc.v[1][p]);
      acc.v[1][p] = make_float2(0.f, 0.f);
    }
    return;
  } else {
#pragma unroll kUnroll
    for (int j = 0; j < kColTile; ++j) {
      const float4 d = stx[j];  // {-t', -t', -x, -y}
      const float2 ct = make_float2(d.x, d.y);
      const int col = c0 + j;
      float2 cx, cy, bj, bj2, cr, dref;
      if (kTrig) cr = make_float2(srt[j], srt[j]);  // -t (stored)
      if (KIND == 0) {
        const float4 c = sxs[j];  // {-s x, -s x, -s y, -s y}
        cx = make_float2(c.x, c.y);
        cy = make_float2(c.z, c.w);
      } else {
        cx = make_float2(d.z, d.z);
        cy = make_float2(d.w, d.w);
      }
      if (KIND == 1 || KIND == 3) {
        dref = add2(SREF, cr);  // t_ref - t_n' >= 0
        if (kC1) bj = mul2(dref, WN);
        if (kC2) bj2 = mul2(dref, WN2);
      }
#pragma unroll
      for (int p = 0; p < kPairs; ++p) {
        const float2 dx = add2(X[p], cx);
        const float2 dy = add2(Y[p], cy);
        float2 dt = make_float2(0.f, 0.f), dtr = dt;
        if (kNeedDt) dt = add2(T[p], ct);
        if (kNeedDtr) dtr = add2(TR[p], cr);
        if (KIND == 0) {
          const float2 u = mul2(dt, dt);
          const float2 q = fma2(dy, dy, fma2(dx, dx, u));
          const float2 eb = make_float2(ex2(-q.x), ex2(-q.y));
          acc.v[0][p] = acc2(acc.v[0][p], eb);
          if (GRAD) {
            acc.v[2][p] = accfma2(q, eb, acc.v[2][p]);
            acc.v[3][p] = accfma2(u, eb, acc.v[3][p]);
          }
          continue;
        }
        const float2 rho = fma2(dy, dy, mul2(dx, dx));
        if (kBg) {
          const float2 u = mul2(dt, dt);
          const float2 q = fma2(rho, A2, u);
          float2 eb = make_float2(ex2(-q.x), ex2(-q.y));
          if (KIND == 2 && excl) {
            const int ra = row_a0 + 64 * p;
            if (col == ra) eb.x = 0.f;
            if (col == ra + 32) eb.y = 0.f;
          }
          acc.v[0][p] = acc2(acc.v[0][p], eb);
          if (GRAD) {
            acc.v[2][p] = accfma2(q, eb, acc.v[2][p]);
            acc.v[3][p] = accfma2(u, eb, acc.v[3][p]);
          }
        }
        if (kTrig && kC1) {
          float2 arg;
          if (KIND == 2) arg = fma2(rho, CN, mul2(dtr, WN));
          else arg = fma2(rho, CN, bj);
          float2 es = make_float2(ex2(arg.x), ex2(arg.y));
          if (KIND == 2) {
            es.x = (col < LO[2 * p]) ? es.x : 0.f;
            es.y = (col < LO[2 * p + 1]) ? es.y : 0.f;
          }
          acc.v[1][p] = acc2(acc.v[1][p], es);
          if (GRAD) {
            acc.v[4][p] = accfma2(rho, es, acc.v[4][p]);
            // separable kinds: the column part t_ref - t_n' of dt (the caller adds t_n - t_ref)
            acc.v[5][p] = accfma2(KIND == 2 ? dtr : dref, es, acc.v[5][p]);
          }
        }
        if (kTrig && kC2) {
          float2 arg2;
          if (KIND == 2) arg2 = fma2(rho, CN2, mul2(dtr, WN2));
          else arg2 = fma2(rho, CN2, bj2);
          float2 es2 = make_float2(ex2(arg2.x), ex2(arg2.y));
          if (KIND == 2) {
            es2.x = (col < LO[2 * p]) ? es2.x : 0.f;
            es2.y = (col < LO[2 * p + 1]) ? es2.y : 0.f;
          }
          acc.v[S2][p] = acc2(acc.v[S2][p], es2);
          if (GRAD) {
            acc.v[S2 + 1][p] = accfma2(rho, es2, acc.v[S2 + 1][p]);
            acc.v[S2 + 2][p] = accfma2(KIND == 2 ? dtr : dref, es2, acc.v[S2 + 2][p]);
          }
        }
      }
    }
  }
}

// A sum v >= 0 into a fixed-point accumulator: round(v 2^F) as an integer (scale = 2^F), so that
// the totals are exact and independent of the order of the additions. A value outside the range
// (not finite, or |v 2^F| >= 2^62) is not added and sets the CTA's flag *bad (shared memory; the
// request's results then become NaN).
__device__ __forceinline__ void red_fix(long long *p, float v, float scale, int *bad) {
  const float x = v * scale;
  if (x == 0.f) return;
  if (!(fabsf(x) < 0x1p62f)) { *bad = 1; return; }
  atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)__float2ll_rn(x));
}
__device__ __forceinline__ void red_fix(long long *p, double v, double scale, int *bad) {
  const double x = v * scale;
  if (x == 0.0) return;
  if (!(fabs(x) < 0x1p62)) { *bad = 1; return; }
  atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)__double2ll_rn(x));
}
// 2^e as a double (|e| <= 1000) and as a float (|e| <= 126), from the exponent bits.
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// A far column tile (background terms only, see SymPlan in hk_internal.h) against this warp's
// rows, each term serving its row and its column; columns are taken in pairs (a, b) = (2m, 2m + 1).
// The tile is staged in pair
// layout (store_cols_pairs): sC[m] = {-s x_a, -s x_b, -s y_a, -s y_b} and, in the time array read
// as float2, {-t'_a, -t'_b}; the swapped pair (b, a) is formed in registers from the same loads
// (a second staged copy cost a third shared load per step, and loglik 3.5% of its time). A
// packed row pair (r0, r1) meets a column
// pair in two packed evaluations, e1 = (e(r0, a), e(r1, b)) and e2 = (e(r0, b), e(r1, a)): both
// add to the row pair's sums as they are, and column a collects e1.x + e2.y, column b
// e1.y + e2.x. Lane L owns column pair L of a 64-column chunk and at step k takes pair
// (L + k) mod 32, so each step covers 2 row pairs x 1 column pair = 8 unordered pairs (16 terms);
// the step's shares of the pair's column sums (over the lane's four rows) go by shuffle to the
// owner, which receives from lane (L - k) mod 32, and after 32 steps each owner adds its pair's
// sums over the warp's 128 rows to fixsum (S_b, Q and T_b: rows 0, 2 and 3). Every sum is formed
// in a fixed order. Per step and
// lane (with the gradient): 49 packed and 6 scalar float32 operations, 8 ex2, 2 shared loads, 6
// shuffles, against 72 packed operations for the same 16 terms row by row.
template <bool GRAD, int NS>
__device__ __forceinline__ void tile_pass_sym_pairs(const float4 *__restrict__ sC, const float4 *__restrict__ sT,
                                                    const float2 (&XS)[kPairs], const float2 (&YS)[kPairs],
                                                    const float2 (&T)[kPairs], Acc32<NS> &acc,
                                                    long long *__restrict__ fixsum, int npad, int c0, float fix_scale,
                                                    int *bad) {
  constexpr int kSymUnroll = GRAD ? HK_SYM_UNROLL : HK_SYM_UNROLL_LL;
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int h = 0; h < kColTile / 64; ++h) {
    float2 cs = make_float2(0.f, 0.f), cq = cs, cu = cs;  // the owned pair's column sums
#pragma unroll kSymUnroll
    for (int k = 0; k < 32; ++k) {
      const int m = h * 32 + ((lane + k) & 31);
      const float4 C = sC[m];
      const float2 T2 = reinterpret_cast<const float2 *>(sT)[m];
      const float2 cx[2] = {make_float2(C.x, C.y), make_float2(C.y, C.x)};
      const float2 cy[2] = {make_float2(C.z, C.w), make_float2(C.w, C.z)};
      const float2 ct[2] = {make_float2(T2.x, T2.y), make_float2(T2.y, T2.x)};
      float2 ps[2], pq[2], pu[2];  // per variant, summed over the row pairs
#pragma unroll
      for (int p = 0; p < kPairs; ++p)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const float2 dx = add2(XS[p], cx[v]), dy = add2(YS[p], cy[v]), dt = add2(T[p], ct[v]);
          const float2 u = mul2(dt, dt);
          const float2 q = fma2(dy, dy, fma2(dx, dx, u));
          const float2 e = make_float2(ex2(-q.x), ex2(-q.y));
          acc.v[0][p] = acc2(acc.v[0][p], e);
          if (GRAD) {
            acc.v[2][p] = accfma2(q, e, acc.v[2][p]);
            acc.v[3][p] = accfma2(u, e, acc.v[3][p]);
          }
          if (p == 0) {
            ps[v] = e;
            if (GRAD) {
              pq[v] = mul2(q, e);
              pu[v] = mul2(u, e);
            }
          } else {
            ps[v] = acc2(ps[v], e);
            if (GRAD) {
              pq[v] = fma2(q, e, pq[v]);
              pu[v] = fma2(u, e, pu[v]);
            }
          }
        }
      const int dst = (lane - k) & 31;  // the lane whose share of this lane's own pair comes now
      cs = add2(cs, make_float2(__shfl_sync(0xffffffffu, ps[0].x + ps[1].y, dst),
                                __shfl_sync(0xffffffffu, ps[0].y + ps[1].x, dst)));
      if (GRAD) {
        cq = add2(cq, make_float2(__shfl_sync(0xffffffffu, pq[0].x + pq[1].y, dst),
                                  __shfl_sync(0xffffffffu, pq[0].y + pq[1].x, dst)));
        cu = add2(cu, make_float2(__shfl_sync(0xffffffffu, pu[0].x + pu[1].y, dst),
                                  __shfl_sync(0xffffffffu, pu[0].y + pu[1].x, dst)));
      }
    }
    long long *f = fixsum + (size_t)c0 + 2 * (h * 32 + lane);
    red_fix(f, cs.x, fix_scale, bad);
    red_fix(f + 1, cs.y, fix_scale, bad);
    if (GRAD) {
      red_fix(f + 2 * (size_t)npad, cq.x, fix_scale, bad);
      red_fix(f + 2 * (size_t)npad + 1, cq.y, fix_scale, bad);
      red_fix(f + 3 * (size_t)npad, cu.x, fix_scale, bad);
      red_fix(f + 3 * (size_t)npad + 1, cu.y, fix_scale, bad);
    }
  }
}

// A shared near column tile (SymPlan, R.sym == 2): the column tile lies before this row tile,
// within the trigger's reach, and each background term serves its row and its column as in the
// far pass, while the trigger terms serve the rows only (the columns are the earlier events).
// Pair layout (store_cols_near): sN[m] = {-x_a, -x_b, -y_a, -y_b} (stored coordinates) and
// sN[kThreads + m] = {-t'_a, -t'_b, -t_a, -t_b} (scaled and stored times). The terms take the
// row-by-row kinds' forms, q = a2 r^2 + dt'^2 and the trigger's r^2 from the stored coordinates.
// BG: background terms, shared (their column shares reach fixsum rows 0, 2 and 3 as in
// tile_pass_sym_pairs). COMP: the trigger components formed (bit 0: component 1 with CN, WN;
// bit 1: component 2 with CN2, WN2, into the sums after the single-kernel ones; 0: none);
// separable (the column factor WN (t_ref - t_n') with t_ref = SREF, the caller applies the row
// factor) unless MASK, which forms WN (t_n - t_n') per pair and keeps the terms with n' < lo(n)
// (ties with a row).
template <bool GRAD, int MIX, bool BG, int COMP, bool MASK>
__device__ __forceinline__ void tile_pass_sym_near(const float4 *__restrict__ sN, const float2 (&X)[kPairs],
                                                   const float2 (&Y)[kPairs], const float2 (&T)[kPairs],
                                                   const float2 (&TR)[kPairs], const int (&LO)[kRowsPerThread],
                                                   int c0, float2 A2, float2 CN, float2 WN, float2 CN2, float2 WN2,
                                                   float2 SREF, Acc32<num_sums(GRAD, MIX)> &acc,
                                                   long long *__restrict__ fixsum, int npad, float fix_scale, int *bad) {
  constexpr int kNearUnroll = GRAD ? HK_NEAR_UNROLL : HK_NEAR_UNROLL_LL;
  constexpr int S2 = GRAD ? 6 : 2;  // component 2's trigger sums
  constexpr bool kC1 = (COMP & 1) != 0, kC2 = MIX > 1 && (COMP & 2) != 0, TRIG = kC1 || kC2;
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int h = 0; h < kColTile / 64; ++h) {
    float2 cs = make_float2(0.f, 0.f), cq = cs, cu = cs;  // the owned pair's column sums (BG)
#pragma unroll kNearUnroll
    for (int k = 0; k < 32; ++k) {
      const int m = h * 32 + ((lane + k) & 31);
      const float4 C = sN[m], D = sN[kThreads + m];
      const float2 cx[2] = {make_float2(C.x, C.y), make_float2(C.y, C.x)};
      const float2 cy[2] = {make_float2(C.z, C.w), make_float2(C.w, C.z)};
      const float2 ct[2] = {make_float2(D.x, D.y), make_float2(D.y, D.x)};
      const float2 cr[2] = {make_float2(D.z, D.w), make_float2(D.w, D.z)};  // -t (stored)
      float2 dref[2], bj[2], bj2[2];
      if (TRIG && !MASK) {
        dref[0] = add2(SREF, cr[0]);  // t_ref - t_n' >= 0
        dref[1] = make_float2(dref[0].y, dref[0].x);
        if (kC1) {
          bj[0] = mul2(dref[0], WN);
          bj[1] = make_float2(bj[0].y, bj[0].x);
        }
        if (kC2) {
          bj2[0] = mul2(dref[0], WN2);
          bj2[1] = make_float2(bj2[0].y, bj2[0].x);
        }
      }
      float2 ps[2], pq[2], pu[2];  // per variant, summed over the row pairs (BG)
#pragma unroll
      for (int p = 0; p < kPairs; ++p)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const float2 dx = add2(X[p], cx[v]), dy = add2(Y[p], cy[v]);
          const float2 rho = fma2(dy, dy, mul2(dx, dx));
          if (BG) {
            const float2 dt = add2(T[p], ct[v]);
            const float2 u = mul2(dt, dt);
            const float2 q = fma2(rho, A2, u);
            const float2 e = make_float2(ex2(-q.x), ex2(-q.y));
            acc.v[0][p] = acc2(acc.v[0][p], e);
            if (GRAD) {
              acc.v[2][p] = accfma2(q, e, acc.v[2][p]);
              acc.v[3][p] = accfma2(u, e, acc.v[3][p]);
            }
            if (p == 0) {
              ps[v] = e;
              if (GRAD) {
                pq[v] = mul2(q, e);
                pu[v] = mul2(u, e);
              }
            } else {
              ps[v] = acc2(ps[v], e);
              if (GRAD) {
                pq[v] = fma2(q, e, pq[v]);
                pu[v] = fma2(u, e, pu[v]);
              }
            }
          }
          if (TRIG) {
            // variant 0 pairs the rows with (a, b), variant 1 with (b, a)
            const int ca = c0 + 2 * m;
            const bool keep_x = !MASK || ca + v < LO[2 * p], keep_y = !MASK || ca + 1 - v < LO[2 * p + 1];
            float2 dtr;
            if (MASK) dtr = add2(TR[p], cr[v]);
            if (kC1) {
              const float2 arg = MASK ? fma2(rho, CN, mul2(dtr, WN)) : fma2(rho, CN, bj[v]);
              float2 es = make_float2(ex2(arg.x), ex2(arg.y));
              if (MASK) {
                es.x = keep_x ? es.x : 0.f;
                es.y = keep_y ? es.y : 0.f;
              }
              acc.v[1][p] = acc2(acc.v[1][p], es);
              if (GRAD) {
                acc.v[4][p] = accfma2(rho, es, acc.v[4][p]);
                acc.v[5][p] = accfma2(MASK ? dtr : dref[v], es, acc.v[5][p]);
              }
            }
            if (kC2) {
              const float2 arg2 = MASK ? fma2(rho, CN2, mul2(dtr, WN2)) : fma2(rho, CN2, bj2[v]);
              float2 es2 = make_float2(ex2(arg2.x), ex2(arg2.y));
              if (MASK) {
                es2.x = keep_x ? es2.x : 0.f;
                es2.y = keep_y ? es2.y : 0.f;
              }
              acc.v[S2][p] = acc2(acc.v[S2][p], es2);
              if (GRAD) {
                acc.v[S2 + 1][p] = accfma2(rho, es2, acc.v[S2 + 1][p]);
                acc.v[S2 + 2][p] = accfma2(MASK ? dtr : dref[v], es2, acc.v[S2 + 2][p]);
              }
            }
          }
        }
      if (BG) {
        const int dst = (lane - k) & 31;
        cs = add2(cs, make_float2(__shfl_sync(0xffffffffu, ps[0].x + ps[1].y, dst),
                                  __shfl_sync(0xffffffffu, ps[0].y + ps[1].x, dst)));
        if (GRAD) {
          cq = add2(cq, make_float2(__shfl_sync(0xffffffffu, pq[0].x + pq[1].y, dst),
                                    __shfl_sync(0xffffffffu, pq[0].y + pq[1].x, dst)));
          cu = add2(cu, make_float2(__shfl_sync(0xffffffffu, pu[0].x + pu[1].y, dst),
                                    __shfl_sync(0xffffffffu, pu[0].y + pu[1].x, dst)));
        }
      }
    }
    if (BG) {
      long long *f = fixsum + (size_t)c0 + 2 * (h * 32 + lane);
      red_fix(f, cs.x, fix_scale, bad);
      red_fix(f + 1, cs.y, fix_scale, bad);
      if (GRAD) {
        red_fix(f + 2 * (size_t)npad, cq.x, fix_scale, bad);
        red_fix(f + 2 * (size_t)npad + 1, cq.y, fix_scale, bad);
        red_fix(f + 3 * (size_t)npad, cu.x, fix_scale, bad);
        red_fix(f + 3 * (size_t)npad + 1, cu.y, fix_scale, bad);
      }
    }
  }
}

// Exact-zero gaps in scaled time dt' between a warp's earliest row and a tile's latest
// column: past kBgZeroGap every background exponent exceeds 130 (ex2 flushes 2^-130 to
// zero); past kTrigZeroExp / -wn every trigger row factor 2^(wn dt') is below 2^-131.
// One percent of margin covers the float32 rounding of the differences.
constexpr float kBgZeroGap = 11.5157f;    // 1.01 * sqrt(130)
constexpr float kTrigZeroExp = 132.31f;   // 1.01 * 131

// Each thread stages kStage columns of a tile: raw values are loaded into registers one
// tile ahead, then scaled, negated and (for packed operands) duplicated into shared memory.
constexpr int kStage = kColTile / kThreads;
static_assert(kColTile % kThreads == 0, "column tile must be a multiple of the CTA width");
static_assert(kColTile == 2 * kThreads, "pair staging of far tiles: one column pair per thread");

struct RawCols {
  float x[kStage], y[kStage], t[kStage];
};

__device__ __forceinline__ RawCols load_cols(const SetView &S, int ct, int tid) {
  RawCols r;
#pragma unroll
  for (int h = 0; h < kStage; ++h) {
    const int j = ct * kColTile + tid + h * kThreads;
    r.x[h] = __ldg(S.x32 + j);
    r.y[h] = __ldg(S.y32 + j);
    r.t[h] = __ldg(S.t32 + j);
  }
  return r;
}

// v * (hi + lo) rounded once (to about 2^-48 of the exact product with the float64 scale).
__device__ __forceinline__ float scale_split(float v, float hi, float lo) { return __fmaf_rn(v, hi, __fmul_rn(v, lo)); }

// Scales of one request: beta for times, s for the coordinates of background-only tiles.
struct Scales {
  float b_hi, b_lo, s_hi, s_lo;
};

// srt[j] = -t_j, the stored time (padded events hold t_N, so differences stay finite).
__device__ __forceinline__ void store_cols(const RawCols &r, int ct, int tid, int n, float t_origin, const Scales &k,
                                           float4 *sxs, float4 *stx, float *srt) {
#pragma unroll
  for (int h = 0; h < kStage; ++h) {
    const int jj = tid + h * kThreads, j = ct * kColTile + jj;
    const float sj = j < n ? scale_split(r.t[h] - t_origin, k.b_hi, k.b_lo) : kPadScaled;
    const float xs = scale_split(r.x[h], k.s_hi, k.s_lo), ys = scale_split(r.y[h], k.s_hi, k.s_lo);
    sxs[jj] = make_float4(-xs, -xs, -ys, -ys);
    stx[jj] = make_float4(-sj, -sj, -r.x[h], -r.y[h]);
    srt[jj] = -r.t[h];
  }
}

// Pair-layout staging of a far tile (tile_pass_sym_pairs): thread tid loads columns 2 tid and
// 2 tid + 1 and writes pair tid of the tile.
__device__ __forceinline__ RawCols load_cols_pairs(const SetView &S, int ct, int tid) {
  RawCols r;
  const int j = ct * kColTile + 2 * tid;
  const float2 x = __ldg(reinterpret_cast<const float2 *>(S.x32 + j));
  const float2 y = __ldg(reinterpret_cast<const float2 *>(S.y32 + j));
  const float2 t = __ldg(reinterpret_cast<const float2 *>(S.t32 + j));
  r.x[0] = x.x; r.x[1] = x.y;
  r.y[0] = y.x; r.y[1] = y.y;
  r.t[0] = t.x; r.t[1] = t.y;
  return r;
}

__device__ __forceinline__ void store_cols_pairs(const RawCols &r, int ct, int tid, int n, float t_origin,
                                                 const Scales &k, float4 *sC, float4 *sT) {
  const int j = ct * kColTile + 2 * tid;
  const float ta = j < n ? scale_split(r.t[0] - t_origin, k.b_hi, k.b_lo) : kPadScaled;
  const float tb = j + 1 < n ? scale_split(r.t[1] - t_origin, k.b_hi, k.b_lo) : kPadScaled;
  const float xa = scale_split(r.x[0], k.s_hi, k.s_lo), xb = scale_split(r.x[1], k.s_hi, k.s_lo);
  const float ya = scale_split(r.y[0], k.s_hi, k.s_lo), yb = scale_split(r.y[1], k.s_hi, k.s_lo);
  sC[tid] = make_float4(-xa, -xb, -ya, -yb);
  reinterpret_cast<float2 *>(sT)[tid] = make_float2(-ta, -tb);
}

// Pair-layout staging of a shared near tile (tile_pass_sym_near), from load_cols_pairs: the stored
// coordinates of pair tid, then its scaled and stored times.
__device__ __forceinline__ void store_cols_near(const RawCols &r, int ct, int tid, int n, float t_origin,
                                                const Scales &k, float4 *sN) {
  const int j = ct * kColTile + 2 * tid;
  const float ta = j < n ? scale_split(r.t[0] - t_origin, k.b_hi, k.b_lo) : kPadScaled;
  const float tb = j + 1 < n ? scale_split(r.t[1] - t_origin, k.b_hi, k.b_lo) : kPadScaled;
  sN[tid] = make_float4(-r.x[0], -r.x[1], -r.y[0], -r.y[1]);
  sN[kThreads + tid] = make_float4(-ta, -tb, -r.t[0], -r.t[1]);
}

// This thread's row coordinates (rows ra = wa + lane + 32 k, packed in pairs k, k + 1),
// stored values or scaled by s with the columns' rounding, so that dx = 0 on the diagonal.
template <bool SCALED>
__device__ __forceinline__ void row_coords(const SetView &S, int ra0, const Scales &k, float2 (&X)[kPairs],
                                           float2 (&Y)[kPairs]) {
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    const int ra = ra0 + 64 * p, rb = ra + 32;
    float xa = __ldg(S.x32 + ra), xb = __ldg(S.x32 + rb), ya = __ldg(S.y32 + ra), yb = __ldg(S.y32 + rb);
    if (SCALED) {
      xa = scale_split(xa, k.s_hi, k.s_lo); xb = scale_split(xb, k.s_hi, k.s_lo);
      ya = scale_split(ya, k.s_hi, k.s_lo); yb = scale_split(yb, k.s_hi, k.s_lo);
    }
    X[p] = make_float2(xa, xb);
    Y[p] = make_float2(ya, yb);
  }
}

// This thread's stored row times (tiles with trigger terms; padded rows hold t_N).
__device__ __forceinline__ void row_times(const SetView &S, int ra0, float2 (&TR)[kPairs]) {
#pragma unroll
  for (int p = 0; p < kPairs; ++p) TR[p] = make_float2(__ldg(S.t32 + ra0 + 64 * p), __ldg(S.t32 + ra0 + 64 * p + 32));
}

// CTA-wide barrier; a single-warp CTA only needs the warp to converge.
__device__ __forceinline__ void cta_sync() {
  if (kThreads == 32) __syncwarp();
  else __syncthreads();
}

// One pair item: the row sums of row tile it.rt over column tiles [c_begin, c_end), then
// (fused) the row tile's merge tree and, in the CTA that completes it, the tile's epilogue;
// otherwise the sums go to the item's partial-sum slot.
// The epilogue of row tile I (Section 2.1, Eq. 1): every event's row sums, get(s, k) for sum s of
// this thread's row k (rows warp * kWarpRows + lane + 32 k); then log lambda_n, the moment ratios
// and the fixed-order reductions (hk_internal.h). Called by every thread of the CTA.
// Event i's terms from its row sums as the pair kernel accumulates them: R_b from Q and T_b, U_s
// from units of time to scaled time, then row_terms.
template <bool GRAD, int MIX, class LogF = StdLog, bool FAST_RCP = false>
__device__ __forceinline__ void row_from_sums(const Request &R, const MixConst &M2, int i, double *sums, double *v) {
  if (GRAD) {
    const double to_scaled = 1.0 / R.tscale;   // beta
    sums[2] = (sums[2] - sums[3]) * R.inv_a2;  // R_b from Q and T_b
    sums[5] *= to_scaled;                      // U_s: from units of time to scaled time
    if (MIX > 1) sums[8] *= to_scaled;
  }
  row_terms<GRAD, MIX, LogF, FAST_RCP>(R, M2, i, sums, v);
}

template <bool GRAD, int MIX, class Get>
__device__ void rowtile_epilogue(const Request &R, const MixConst &M2, int I, Get get) {
  constexpr int NS = num_sums(GRAD, MIX);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = R.set.n;
  double v[GRAD ? 1 + NS : 1] = {};
#pragma unroll
  for (int k = 0; k < kRowsPerThread; ++k) {
    const int i = I * kRowTile + warp * kWarpRows + lane + 32 * k;
    if (i < n) {
      double sums[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) sums[s] = get(s, k);
      row_from_sums<GRAD, MIX>(R, M2, i, sums, v);
    }
  }
  rowtile_reduce<GRAD, MIX>(R, M2, I, v);
}

template <bool GRAD, int MIX>
__device__ void run_piece(const Batch &B, const Request &R, const PairItem &it, int c_begin, int c_end,
                          const SymPlan &plan, float4 (*sxs)[kColTile], float4 (*stx)[kColTile],
                          float (*srt)[kColTile], double *sacc) {
  constexpr int NS = num_sums(GRAD, MIX);
  constexpr int S2 = GRAD ? 6 : 2;  // component 2's trigger sums (mixture)
  const SetView &S = R.set;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int row0 = it.rt * kRowTile;
  const float t_origin = S.t32[row0];
  // tile classes: the trigger component reaching furthest (the larger wn, both are negative)
  const float wn = MIX > 1 ? fmaxf(R.wn, B.mix2.wn2) : R.wn;
  const Scales sk{R.beta, R.beta_lo, R.s_hi, R.s_lo};
  const int n = S.n;
  const int wa = row0 + warp * kWarpRows, wb = wa + kWarpRows - 1;
  const int lo_wa = S.lo32[wa], lo_wb = S.lo32[wb];
  const bool excl = (R.flags & 1) != 0;
  const int row_a0 = wa + lane;

  float2 T[kPairs];
  int LO[kRowsPerThread];
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    const int ra = row_a0 + 64 * p, rb = ra + 32;
    T[p] = make_float2(ra < n ? scale_split(S.t32[ra] - t_origin, sk.b_hi, sk.b_lo) : kPadScaled,
                       rb < n ? scale_split(S.t32[rb] - t_origin, sk.b_hi, sk.b_lo) : kPadScaled);
    LO[2 * p] = S.lo32[ra];
    LO[2 * p + 1] = S.lo32[rb];
  }
  // row coordinates are reloaded (L1) per tile, scaled for the background-only kinds and stored
  // for the others, so that no kind holds the other's registers
  float2 XS[kPairs], YS[kPairs];
  const float2 A2 = make_float2(R.a2, R.a2), CN = make_float2(R.cn, R.cn);
  const float2 CN2 = make_float2(B.mix2.cn2, B.mix2.cn2);
  // trigger slopes per unit of stored time, -omega log2(e) rounded once (formed in the tiles with
  // trigger terms, from the launch parameters, so that they hold no register elsewhere)
  auto slope = [&](double omega) {
    const float w = (float)(-omega * kLog2eD);
    return make_float2(w, w);
  };
  // row factor 2^(WN (t_n - t_ref)) of a separable trigger tile (each component's own, for the
  // components in comps); U_s gets the row part of dt = (t_n - t_ref) + (t_ref - t_n'), both >= 0
  auto row_factor = [&](float sref, float2 WN, float2 WN2, int comps, const float2 (&TR)[kPairs], Acc32<NS> &acc) {
    const float2 sr = make_float2(-sref, -sref);
#pragma unroll
    for (int p = 0; p < kPairs; ++p) {
      const float2 d = __fadd2_rn(TR[p], sr);
      if (MIX == 1 || (comps & 1)) {
        const float2 w = __fmul2_rn(d, WN);
        const float2 a = make_float2(ex2(w.x), ex2(w.y));
        if (GRAD) {
          acc.v[5][p] = __fmul2_rn(__ffma2_rn(d, acc.v[1][p], acc.v[5][p]), a);
          acc.v[4][p] = __fmul2_rn(acc.v[4][p], a);
        }
        acc.v[1][p] = __fmul2_rn(acc.v[1][p], a);
      }
      if (MIX > 1 && (comps & 2)) {
        const float2 w2 = __fmul2_rn(d, WN2);
        const float2 a2 = make_float2(ex2(w2.x), ex2(w2.y));
        if (GRAD) {
          acc.v[S2 + 2][p] = __fmul2_rn(__ffma2_rn(d, acc.v[S2][p], acc.v[S2 + 2][p]), a2);
          acc.v[S2 + 1][p] = __fmul2_rn(acc.v[S2 + 1][p], a2);
        }
        acc.v[S2][p] = __fmul2_rn(acc.v[S2][p], a2);
      }
    }
  };
  const float s_first = __shfl_sync(0xffffffffu, T[0].x, 0);            // scaled time of the warp's
  const float s_last = __shfl_sync(0xffffffffu, T[kPairs - 1].y, 31);  // first and last rows

  __shared__ int s_bad;  // with R.sym: a sum of this item left the fixed-point range (red_fix)
  if (tid == 0) s_bad = 0;
  if (R.sym) cta_sync();

  // float64 row accumulators live in shared memory, one slot per (sum, row, thread)
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) sacc[(s * kRowsPerThread + k) * kThreads + tid] = 0.0;

  // far tiles are staged in pair layout (tile_pass_sym_pairs), shared near ones in their own pair
  // layout (tile_pass_sym_near), the rest one column at a time (tile_pass)
  auto layout = [&](int c) {
    return R.sym && c < plan.sym_end ? 1 : c >= plan.sym_end && c < plan.near_end ? 2 : 0;
  };
  auto load = [&](int c, int lay) { return lay ? load_cols_pairs(S, c, tid) : load_cols(S, c, tid); };
  auto stage = [&](const RawCols &r, int c, int lay, int b) {
    if (lay == 1) store_cols_pairs(r, c, tid, n, t_origin, sk, sxs[b], stx[b]);
    else if (lay == 2) store_cols_near(r, c, tid, n, t_origin, sk, sxs[b]);
    else store_cols(r, c, tid, n, t_origin, sk, sxs[b], stx[b], srt[b]);
  };
  int ct = c_begin;
  if (ct < c_end) {  // an empty slice of the window writes zero partial sums
    const int lay = layout(ct);
    stage(load(ct, lay), ct, lay, 0);
    cta_sync();
  }
  for (int k = 0; ct < c_end; ++ct, ++k) {
    const int buf = k & 1;
    const bool has_next = ct + 1 < c_end;
    const int next_lay = layout(ct + 1);
    RawCols nxt;
    if (has_next) nxt = load(ct + 1, next_lay);
    const int c0 = ct * kColTile, c1 = c0 + kColTile;
    int kind, comps = 1;  // comps: the mixture components with nonzero trigger terms (bit mask)
    if (R.sym && ct < plan.sym_end) {  // far: background only, shared with the columns' rows
      const float gap = s_first + reinterpret_cast<const float2 *>(stx[buf])[kColTile / 2 - 1].y;  // the latest column
      kind = gap >= kBgZeroGap ? -1 : 4;
    } else if (ct < plan.near_end) {  // shared near tile: the same classes as below
      if (c1 <= lo_wa) {
        const float gap = s_first + sxs[buf][kColTile - 1].y;  // t'(first row) - t'(latest column)
        const bool bg_zero = gap >= kBgZeroGap, trig_zero = wn * gap <= -kTrigZeroExp;
        kind = bg_zero ? (trig_zero ? -1 : 7) : (trig_zero ? 5 : 6);
        if (MIX > 1)
          comps = (R.wn * gap <= -kTrigZeroExp ? 0 : 1) | (B.mix2.wn2 * gap <= -kTrigZeroExp ? 0 : 2);
      } else {
        kind = 8;  // a column tied with a row of this warp
      }
    } else if (c1 <= lo_wa) {  // every pair causal: which of the two terms can be nonzero?
      const float gap = s_first + stx[buf][kColTile - 1].x;  // t'(first row) - t'(latest column)
      const bool bg_zero = gap >= kBgZeroGap, trig_zero = wn * gap <= -kTrigZeroExp;
      kind = bg_zero ? (trig_zero ? -1 : 3) : (trig_zero ? 0 : 1);
      if (MIX > 1)
        comps = (R.wn * gap <= -kTrigZeroExp ? 0 : 1) | (B.mix2.wn2 * gap <= -kTrigZeroExp ? 0 : 2);
    } else if (c0 >= lo_wb) {  // no causal pair: background only, zero past its reach
      const float gap = -stx[buf][0].x - s_last;  // t'(earliest column) - t'(last row)
      kind = gap >= kBgZeroGap ? -1 : 0;
    } else {
      kind = 2;
    }
    if (excl && c0 <= wb && c1 > wa) kind = 2;
    Acc32<NS> acc;
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int p = 0; p < kPairs; ++p) acc.v[s][p] = make_float2(0.f, 0.f);
    float2 X[kPairs], Y[kPairs], TR[kPairs];  // stored row coordinates and times, tiles with trigger terms
    if (kind == 0) {
      row_coords<true>(S, row_a0, sk, XS, YS);
      tile_pass<0, GRAD, MIX>(sxs[buf], stx[buf], srt[buf], XS, YS, T, T, LO, row_a0, c0, excl, A2, CN, CN, CN2, CN2,
                              CN, acc);
    } else if (kind == 4) {
      row_coords<true>(S, row_a0, sk, XS, YS);
      tile_pass_sym_pairs<GRAD>(sxs[buf], stx[buf], XS, YS, T, acc, R.fixsum, S.npad, c0, pow2f(R.fix_bits[0]),
                                &s_bad);
    } else if (kind >= 5) {
      row_coords<false>(S, row_a0, sk, X, Y);
      const float2 WN = slope(R.omega), WN2 = MIX > 1 ? slope(B.mix2.omega2) : WN;
      const float sref = -sxs[buf][kColTile - 1].w;  // t_ref: the tile's latest column (stored time)
      const float2 SREF = make_float2(sref, sref);
      const float fs = pow2f(R.fix_bits[0]);
      auto near = [&](auto bg_c, auto comp_c, auto mask_c) {
        tile_pass_sym_near<GRAD, MIX, decltype(bg_c)::value, decltype(comp_c)::value, decltype(mask_c)::value>(
            sxs[buf], X, Y, T, TR, LO, c0, A2, CN, WN, CN2, WN2, SREF, acc, R.fixsum, S.npad, fs, &s_bad);
      };
      using BY = std::integral_constant<bool, true>;
      using BN = std::integral_constant<bool, false>;
      using C0 = std::integral_constant<int, 0>;
      using C1 = std::integral_constant<int, 1>;
      using C2 = std::integral_constant<int, 2>;
      using CA = std::integral_constant<int, (MIX > 1 ? 3 : 1)>;  // every component
      if (kind == 8) {  // rare (ties across the tile's edge): the background, then the masked trigger
        near(BY{}, C0{}, BN{});
        row_times(S, row_a0, TR);
        near(BN{}, CA{}, BY{});
      } else if (kind == 5) {
        near(BY{}, C0{}, BN{});
      } else {
        if constexpr (MIX == 1) {
          if (kind == 6) near(BY{}, C1{}, BN{});
          else near(BN{}, C1{}, BN{});
        } else if (comps == 3) {
          if (kind == 6) near(BY{}, CA{}, BN{});
          else near(BN{}, CA{}, BN{});
        } else if (comps == 1) {
          if (kind == 6) near(BY{}, C1{}, BN{});
          else near(BN{}, C1{}, BN{});
        } else {
          if (kind == 6) near(BY{}, C2{}, BN{});
          else near(BN{}, C2{}, BN{});
        }
        row_times(S, row_a0, TR);
        row_factor(sref, WN, WN2, comps, TR, acc);
      }
    } else if (kind == 1 || kind == 3) {
      row_coords<false>(S, row_a0, sk, X, Y);
      row_times(S, row_a0, TR);
      const float sref = -srt[buf][kColTile - 1];  // t_ref: the tile's latest column (stored time)
      const float2 SREF = make_float2(sref, sref);
      const float2 WN = slope(R.omega), WN2 = MIX > 1 ? slope(B.mix2.omega2) : WN;
      auto pass = [&](auto kind_c, auto comp_c) {
        tile_pass<decltype(kind_c)::value, GRAD, MIX, decltype(comp_c)::value>(
            sxs[buf], stx[buf], srt[buf], X, Y, T, TR, LO, row_a0, c0, excl, A2, CN, WN, CN2, WN2, SREF, acc);
      };
      using K1 = std::integral_constant<int, 1>;
      using K3 = std::integral_constant<int, 3>;
      using C1 = std::integral_constant<int, 1>;
      using C2 = std::integral_constant<int, 2>;
      using C3 = std::integral_constant<int, 3>;
      if constexpr (MIX == 1) {
        if (kind == 1) pass(K1{}, C1{});
        else pass(K3{}, C1{});
      } else if (comps == 3) {
        if (kind == 1) pass(K1{}, C3{});
        else pass(K3{}, C3{});
      } else if (comps == 1) {
        if (kind == 1) pass(K1{}, C1{});
        else pass(K3{}, C1{});
      } else {
        if (kind == 1) pass(K1{}, C2{});
        else pass(K3{}, C2{});
      }
      row_factor(sref, WN, WN2, comps, TR, acc);
    } else if (kind == 2) {
      row_coords<false>(S, row_a0, sk, X, Y);
      row_times(S, row_a0, TR);
      const float2 WN = slope(R.omega), WN2 = MIX > 1 ? slope(B.mix2.omega2) : WN;
      tile_pass<2, GRAD, MIX, 3>(sxs[buf], stx[buf], srt[buf], X, Y, T, TR, LO, row_a0, c0, excl, A2, CN, WN, CN2,
                                 WN2, WN, acc);
    }  // kind -1: every term of the tile is exactly zero for this warp
    // fold the tile's sums into float64; a tile without trigger (background) terms leaves
    // those sums at zero, so they are skipped
    const bool fold_bg = kind == 0 || kind == 1 || kind == 2 || kind == 4 || kind == 5 || kind == 6 || kind == 8;
    const bool fold_trig = (kind >= 1 && kind <= 3) || kind >= 6;
    if (kind == 2 || kind == 8) comps = 3;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const bool trig_sum = GRAD ? (s == 1 || s >= 4) : s >= 1;  // S_s, R_s, U_s (each component)
      const int comp = s >= (GRAD ? 6 : 2) ? 2 : 1;               // the component of a trigger sum
      if (trig_sum ? !(fold_trig && (MIX == 1 || (comps & comp))) : !fold_bg) continue;
#pragma unroll
      for (int p = 0; p < kPairs; ++p) {
        sacc[(s * kRowsPerThread + 2 * p) * kThreads + tid] += (double)acc.v[s][p].x;
        sacc[(s * kRowsPerThread + 2 * p + 1) * kThreads + tid] += (double)acc.v[s][p].y;
      }
    }
    if (has_next) stage(nxt, ct + 1, next_lay, buf ^ 1);
    cta_sync();
  }
  // this thread's rows: la = warp * kWarpRows + lane + 32 k, sums at sacc[(s R + k) T + tid]
  auto store = [&](int to) {
    double *dst = R.partials + (size_t)to * NS * kRowTile;
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k)
#pragma unroll
      for (int s = 0; s < NS; ++s)
        dst[s * kRowTile + warp * kWarpRows + lane + 32 * k] = sacc[(s * kRowsPerThread + k) * kThreads + tid];
  };
  if (!B.fused) {  // row-tile-major slot of the item's first leaf (unfused launches use 1-leaf items)
    store(it.rt * R.slices + it.node * it.span);
    return;
  }
  if (R.sym) {
    // Every event's sums go to fixsum: this item's far column tiles have added their columns'
    // shares there; now its rows' float64 sums. Sym requests always run in split batches
    // (launch_batch), so the item ends here.
    const size_t np = (size_t)S.npad;
    long long *fx = R.fixsum + row0 + warp * kWarpRows + lane;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const double scale = pow2d(R.fix_bits[s]);
#pragma unroll
      for (int k = 0; k < kRowsPerThread; ++k)
        red_fix(fx + s * np + 32 * k, sacc[(s * kRowsPerThread + k) * kThreads + tid], scale, &s_bad);
    }
    cta_sync();
    if (tid == 0 && s_bad && R.status) atomicOr(R.status, kStatusFixRange);
    return;  // epilogue_fix_kernel, launched after this kernel (Batch::split), finishes every row
  }
  auto merge = [&](int from) {
    const double *src = R.partials + (size_t)from * NS * kRowTile;
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k)
#pragma unroll
      for (int s = 0; s < NS; ++s)
        sacc[(s * kRowsPerThread + k) * kThreads + tid] += __ldcg(src + s * kRowTile + warp * kWarpRows + lane + 32 * k);
  };
  const int root = merge_tree<GRAD>(R, it, store, merge);
  if (root < 0) mark_timeout(R);
  if (root <= 0) return;
  rowtile_epilogue<GRAD, MIX>(R, B.mix2, it.rt,
                              [&](int s, int k) { return sacc[(s * kRowsPerThread + k) * kThreads + tid]; });
}

// sym_plan_scan (hk_internal.h) with the later row tiles taken 32 at a time, one per lane; called
// by one full warp, every lane returns the plan of row tile I.
__device__ SymPlan sym_plan_warp(const Request &R, int I, int2 win) {
  const WinTable &W = R.set.win32;
  const float *t = R.set.t32;
  const int lane = threadIdx.x & 31;
  const SymK own = sym_k(R, W, (double)__ldg(t + (size_t)I * kRowTile));
  // shared near tiles: the plan needs no later row tile (e_col, which no kernel reads, stays 0)
  if (R.sym == 2) return sym_plan_near(win, max(win.x, 2 * own.ib), I, 0);
  int e_col = 0, kmax = I;
  for (int base = I + 1; base < R.set.nrt; base += 32) {
    const int K = base + lane;
    bool done = true;
    if (K < R.set.nrt) {
      const SymK k = sym_k(R, W, (double)__ldg(t + (size_t)K * kRowTile));
      done = sym_done(k, I);
      if (!done) {
        bool near;
        sym_visit(k, I, &e_col, &near);
        if (near) kmax = K;
      }
    }
    if (__any_sync(0xffffffffu, done)) break;  // every later row tile is done too
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    e_col += __shfl_xor_sync(0xffffffffu, e_col, off);
    kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, off));
  }
  const int sym_end = max(win.x, 2 * own.ib);
  return SymPlan{sym_end, sym_end, min(win.y, 2 * kmax + 2), e_col};
}

template <bool GRAD, int MIX>
__global__ void __launch_bounds__(kThreads, MIX > 1 ? (GRAD ? HK_MIN_CTAS_MIX : HK_MIN_CTAS_MIX_LL)
                                                      : GRAD ? HK_MIN_CTAS : HK_MIN_CTAS_LL)
    pair_mixed_kernel(const __grid_constant__ Batch B) {
  constexpr int NS = num_sums(GRAD, MIX);
  // static shared memory, loglik + gradient: 21,944 bytes with the reductions' scratch; ten
  // resident CTAs need at most 22,272 (10 x (22,272 + 1,024 reserved) <= 228 KB in 128-byte units)
  __shared__ __align__(16) float4 sxs[2][kColTile];
  __shared__ __align__(16) float4 stx[2][kColTile];
  __shared__ float srt[2][kColTile];
  __shared__ double sacc[NS * kRowsPerThread * kThreads];
  __shared__ int2 s_win;
  const int item = blockIdx.x;
  const Request &R = B.req[find_request(B, item)];
  const int local = item - R.item_begin, nc = comp_items(R);
  if (local < nc) {  // compensator item of row tile `local`
    compensator_tile<MIX>(R, B.mix2, R.set.t32, local, GRAD);
    if (B.fused && !(B.split && R.sym)) finish_request<GRAD, MIX>(R);
    return;
  }
  const PairItem it = item_at(R, local - nc);
  const int rt = it.rt, ns = R.slices, l0 = it.node * it.span, l1 = min(l0 + it.span, ns);
  int2 w = table_window_rt(R, R.set.win32, R.set.t32, rt);
  if (w.x < 0) {  // no lookup table: one warp searches the times
    if (threadIdx.x < 32) {
      const int2 v = column_window(R, R.set.t32, rt);
      if (threadIdx.x == 0) s_win = v;
    }
    cta_sync();
    w = s_win;
  }
  SymPlan plan{w.x, w.x, w.y, 0};
  if (R.sym) {  // far and near column tiles of this row tile (the host enables sym only with a table)
    __shared__ SymPlan s_plan;
    if (threadIdx.x < 32) {
      const SymPlan v = sym_plan_warp(R, rt, w);
      if (threadIdx.x == 0) s_plan = v;
    }
    cta_sync();
    plan = s_plan;
    w.y = plan.end;
  }
  // leaves: equal shares of the window's cost, a far column tile weighing HK_FAR_WEIGHT / 10 and a
  // shared near one HK_SNEAR_WEIGHT / 10 row-by-row ones (without sym every tile weighs the same)
  const long long fw = R.sym ? HK_FAR_WEIGHT : 10, sw = HK_SNEAR_WEIGHT;
  const long long nf = plan.sym_end - w.x, nsn = plan.near_end - plan.sym_end, nn = w.y - plan.near_end;
  const long long total = nf * fw + nsn * sw + nn * 10;
  auto at = [&](int l) {  // column tile where leaf l starts
    long long pos = total * l / ns;
    if (pos < nf * fw) return w.x + (int)(pos / fw);
    pos -= nf * fw;
    if (pos < nsn * sw) return plan.sym_end + (int)(pos / sw);
    return plan.near_end + (int)((pos - nsn * sw) / 10);
  };
  const int c_begin = at(l0), c_end = at(l1);
  run_piece<GRAD, MIX>(B, R, it, c_begin, c_end, plan, sxs, stx, srt, sacc);
}

// The split epilogue (Batch::split): block b of the batch's sym requests, in request order,
// takes events [b kEpiRows, (b + 1) kEpiRows) of its request, one per thread: the event's sums
// from fixsum, its terms (row_from_sums), a fixed-order reduction of the block, the gradient's
// Theta factors and, in the even block of each row tile, the tile's compensator sums subtracted,
// into rt_sum[b]. The last block of each group of kEpiGroup blocks (a counter per group) sums
// the group in order into a group slot, and the last group of the request (the request's final
// counter) sums the groups in order into ell and the gradient: every sum has a fixed order, and
// the final one reads ceil(blocks / 32) slots instead of every block's. The pair kernel's
// additions to fixsum and its compensator sums are complete when this kernel starts (same
// stream).
// ---- the split epilogue's float64 arithmetic ------------------------------------------------
// GB300's float64 pipe runs about 1.6 operations per clock and SM, and the split epilogue is bound
// by it (a 256-row block of events spends ~57 DADD-equivalents per event, 45% of them CUDA's
// log). Three changes take it to ~25:
// - the fixed-point sums are turned into doubles on the integer pipe (fix_to_double);
// - 1 / lambda from the float32 reciprocal and one Newton step (row_terms' FAST_RCP);
// - the log of lambda by a table-driven method (Tang, "Table-driven implementation of the
//   logarithm function in IEEE floating-point arithmetic", ACM TOMS 16(4), 1990): with
//   x = 2^e m, m in [1, 2), and j the top 7 bits of m's fraction, c_j = 1 / (1 + (j + 1/2) / 128)
//   rounded to float32 and r = m c_j - 1 in one rounding (|r| < 2^-7.9),
//     ln x = e ln 2 + (-ln c_j) + ln(1 + r),  ln(1 + r) = r - r^2/2 + ... + r^7/7
//   (the first dropped term is below 2^-64); -ln c_j comes from a table computed on the host in
//   extended precision (init_log_table), ln 2 in a 40-bit head (e ln2_hi exact) and a tail.
//   About 12 float64 operations against ~27 for CUDA's log, and within a few units in the last
//   place of it (the ell of hawkes_event_terms is checked against the log of its own lambda_i).
__device__ double g_logtab[2 * 128];  // c_j, then -ln c_j
constexpr double kLn2Hi = 0x1.62e42fefa4000p-1, kLn2Lo = -0x1.8432a1b0e2634p-43;

struct TabLog {
  __device__ __forceinline__ double operator()(double x) const {
    const long long b = __double_as_longlong(x);
    const int eb = (int)(b >> 52);
    if (eb <= 0 || eb >= 0x7ff) return log(x);  // zero, negative, subnormal, inf or NaN
    const int j = (int)((b >> 45) & 127);
    const double m = __longlong_as_double((b & 0xfffffffffffffll) | 0x3ff0000000000000ll);
    const double c = __ldg(g_logtab + j), t = __ldg(g_logtab + 128 + j);
    const double r = fma(m, c, -1.0);
    double q = fma(r, 1.0 / 7.0, -1.0 / 6.0);
    q = fma(r, q, 0.2);
    q = fma(r, q, -0.25);
    q = fma(r, q, 1.0 / 3.0);
    q = fma(r, q, -0.5);
    const double p = fma(r * r, q, r);
    const double e = (double)(eb - 1023);
    return fma(e, kLn2Hi, t) + fma(e, kLn2Lo, p);
  }
};

// The double nearest below v 2^-F for a fixed-point sum v (Request::fixsum), from the bits of v
// on the integer pipe: the leading one of |v| sets the exponent, the next 52 bits the mantissa
// (the rest is cut, 2^-53 relative at most), and F only moves the exponent.
__device__ __forceinline__ double fix_to_double(long long v, int F) {
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned long long u = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll((long long)u);
  const unsigned long long m = u << lz;  // leading one at bit 63
  const unsigned long long e = (unsigned long long)(1023 + 63 - lz - F);
  return __longlong_as_double((long long)(sign | (e << 52) | ((m >> 11) & 0xfffffffffffffull)));
}

// Warp totals of P values per lane (P a power of two, at most 32) by a transposing butterfly, in a
// fixed order: at the offsets 16, 8, ... each lane keeps half of its values (the lower half where
// its bit of the offset is 0) and adds its partner's matching half, so the P totals need
// P - 1 + 5 - log2 P additions per lane instead of 5 P for P separate trees (the float64 pipe is
// what bounds the split epilogue). On return lane l holds the total of value l >> (5 - log2 P)
// in x[0] (every lane of a group holds the same bits: the last levels add a + b and b + a).
template <int P>
__device__ __forceinline__ void warp_transpose_sum(double (&x)[P]) {
  static_assert(P >= 1 && P <= 32 && (P & (P - 1)) == 0, "P: a power of two up to 32");
  const int lane = threadIdx.x & 31;
  int o = 16;
#pragma unroll
  for (int m = P; m > 1; m >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < m / 2; ++i) {
      const double send = up ? x[i] : x[m / 2 + i];
      const double keep = up ? x[m / 2 + i] : x[i];
      x[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (; o > 0; o >>= 1) x[0] += __shfl_xor_sync(0xffffffffu, x[0], o);
}

static_assert(kEpiRows <= 32 * kMaxCtaWarps, "reduction scratch too narrow for the split epilogue");
constexpr int kEpiGroup = 32;  // epilogue blocks per first-level group of the final sum

// Sum of `count` slots of NV values (kOut apart) by one full warp, in a fixed order: lane l takes
// slots l, l + 32, ... in turn, then a fixed shuffle tree; lane 0 holds the totals in x.
template <int NV>
__device__ __forceinline__ void warp_sum_slots(const double *slots, int count, double (&x)[NV]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < NV; ++q) x[q] = 0.0;
  for (int c = lane; c < count; c += 32)
#pragma unroll
    for (int q = 0; q < NV; ++q) x[q] += __ldcg(slots + (size_t)c * kOut + q);
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x[q] += __shfl_down_sync(0xffffffffu, x[q], off);
}
template <bool GRAD, int MIX>
__global__ void __launch_bounds__(kEpiRows) epilogue_fix_kernel(const __grid_constant__ Batch B) {
  constexpr int NS = num_sums(GRAD, MIX);
  int b = blockIdx.x, r = 0;
  for (; r < B.nreq; ++r) {
    if (!B.req[r].sym) continue;
    const int nb = epi_blocks(B.req[r]);
    if (b < nb) break;
    b -= nb;
  }
  const Request &R = B.req[r];
  const int i = b * kEpiRows + threadIdx.x;
  double v[GRAD ? 1 + NS : 1] = {};
  if (i < R.set.n) {
    const size_t np = (size_t)R.set.npad;
    double sums[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) sums[s] = fix_to_double(__ldcg(R.fixsum + s * np + i), R.fix_bits[s]);
    row_from_sums<GRAD, MIX, TabLog, true>(R, B.mix2, i, sums, v);
  }
  // block partial: log lambda and the gradient terms (grad_from_moments), less the compensator
  // sums of row tile b / 2 in the even block of the tile, into rt_sum[b]
  constexpr int NV = GRAD ? 1 + num_grad(MIX) : 1;
  constexpr int NR = GRAD ? 1 + NS : 1;
  double *red = reduce_scratch(), *tot = red + kMaxCtaWarps * kRedWidth;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {
    constexpr int P = NR == 1 ? 1 : NR <= 2 ? 2 : NR <= 4 ? 4 : NR <= 8 ? 8 : 16;
    constexpr int SH = P == 1 ? 5 : P == 2 ? 4 : P == 4 ? 3 : P == 8 ? 2 : 1;  // 5 - log2 P
    double x[P];
#pragma unroll
    for (int q = 0; q < P; ++q) x[q] = q < NR ? v[q] : 0.0;
    warp_transpose_sum<P>(x);
    const int q = lane >> SH;
    if ((lane & ((1 << SH) - 1)) == 0 && q < NR) red[warp * kRedWidth + q] = x[0];
  }
  __syncthreads();
  if (tid < NR) {
    double x = 0.0;
    for (int w = 0; w < kEpiRows / 32; ++w) x += red[w * kRedWidth + tid];
    tot[tid] = x;
  }
  __syncthreads();
  const int nblk = epi_blocks(R), ngrp = (nblk + kEpiGroup - 1) / kEpiGroup, g = b / kEpiGroup;
  __shared__ unsigned s_last;
  if (tid == 0) {
    double val[NV];
    val[0] = tot[0];
    if (GRAD) grad_from_moments<MIX>(R, B.mix2, tot + 1, val + 1);
    const bool sub = R.comp && (b & 1) == 0;
#pragma unroll
    for (int q = 0; q < NV; ++q) R.rt_sum[(size_t)b * kOut + q] = sub ? val[q] - R.comp[(size_t)(b / 2) * kOut + q] : val[q];
    __threadfence();
    const unsigned members = (unsigned)min(kEpiGroup, nblk - g * kEpiGroup);
    s_last = atomicAdd(R.rt_count + g, 1u) == members - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  // the last block of group g sums the group's partials in order into slot 2 nrt + g; the last
  // group to finish sums the groups' in order into ell and the gradient
  double *gsum = R.rt_sum + (size_t)2 * R.set.nrt * kOut;
  if (warp == 0) {
    __threadfence();
    double x[NV];
    warp_sum_slots<NV>(R.rt_sum + (size_t)g * kEpiGroup * kOut, min(kEpiGroup, nblk - g * kEpiGroup), x);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < NV; ++q) gsum[(size_t)g * kOut + q] = x[q];
      __threadfence();
      s_last = atomicAdd(R.rt_count + request_counters(R) - 1, 1u) == (unsigned)ngrp - 1u;
    }
    __syncwarp();
    if (__shfl_sync(0xffffffffu, s_last, 0)) {
      __threadfence();
      warp_sum_slots<NV>(gsum, ngrp, x);
      if (lane == 0) {
        // a sum that left the fixed-point range (red_fix) was not added: the results are NaN
        const bool nan = R.status && (__ldcg(R.status) & kStatusFixRange);
#pragma unroll
        for (int q = 0; q < NV; ++q) R.out[q] = nan ? __longlong_as_double(0x7ff8000000000000ll) : x[q];
      }
    }
  }
}

}  // namespace

// The table of TabLog on the current device: c_j = 1 / (1 + (j + 1/2) / 128) rounded to float32,
// and -ln c_j from the host's extended-precision log, rounded once to double.
cudaError_t init_log_table() {
  double tab[2 * 128];
  for (int j = 0; j < 128; ++j) {
    const float c = (float)(1.0 / (1.0 + (j + 0.5) / 128.0));
    tab[j] = (double)c;
    tab[128 + j] = (double)(-logl((long double)c));
  }
  return cudaMemcpyToSymbol(g_logtab, tab, sizeof(tab));
}

cudaError_t launch_epilogue_fix(const Batch &b, bool grad, cudaStream_t s) {
  int blocks = 0;
  for (int r = 0; r < b.nreq; ++r)
    if (b.req[r].sym) blocks += epi_blocks(b.req[r]);
  if (!b.split || blocks == 0) return cudaSuccess;
  if (b.req[0].mix > 1) {
    if (grad) epilogue_fix_kernel<true, 2><<<blocks, kEpiRows, 0, s>>>(b);
    else epilogue_fix_kernel<false, 2><<<blocks, kEpiRows, 0, s>>>(b);
  } else if (grad) {
    epilogue_fix_kernel<true, 1><<<blocks, kEpiRows, 0, s>>>(b);
  } else {
    epilogue_fix_kernel<false, 1><<<blocks, kEpiRows, 0, s>>>(b);
  }
  return cudaGetLastError();
}

cudaError_t launch_pair_mixed(const Batch &b, bool grad, cudaStream_t s) {
  if (b.total_items < 1) return cudaErrorInvalidValue;
  if (b.req[0].mix > 1) {  // a trigger mixture (one request per launch)
    if (grad) pair_mixed_kernel<true, 2><<<b.total_items, kThreads, 0, s>>>(b);
    else pair_mixed_kernel<false, 2><<<b.total_items, kThreads, 0, s>>>(b);
  } else if (grad) {
    pair_mixed_kernel<true, 1><<<b.total_items, kThreads, 0, s>>>(b);
  } else {
    pair_mixed_kernel<false, 1><<<b.total_items, kThreads, 0, s>>>(b);
  }
  return cudaGetLastError();
}

int occupancy_pair_mixed(bool grad) {
  int n = 0;
  if (grad) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_mixed_kernel<true, 1>, kThreads, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_mixed_kernel<false, 1>, kThreads, 0);
  return n;
}

}  // namespace hk
