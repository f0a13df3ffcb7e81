// Grouped mixed-precision pair kernel: up to G requests on one event set per CTA (G = 4 with
// the gradient, 8 for the log-likelihood alone).
//
// A batch of K parameter vectors on one set (Section 2.2: many MH chains, or one chain's
// proposals) shares every pair's geometry. For each (row n, column n') the CTA forms once
//   dx, dy, r^2 = dx^2 + dy^2, dt = t_n - t_n' (days, the difference of the stored float32
//   times, rounded once: exact where t_n' >= t_n / 2), dt^2
// and then, for each request k of its group, the terms of Section 2.1, Eq. 1 from those:
//   e_b = 2^-(a2_k r^2 + b2_k dt^2),  a2 = log2(e)/(2 tau_x^2), b2 = log2(e)/(2 tau_t^2)
//   e_s = 2^(cn_k r^2 + wn_k dt),     cn = -log2(e)/(2 h^2),    wn = -omega log2(e)
// with the same row sums as the single-request kernel (S_b, S_s, R_b, T_b, R_s, U_s), the
// moments in raw units (r^2 in km^2, dt in days). Shared work per pair: 6 float32 operations;
// per request and background term: 5 (exponent 2, sum, 2 moments), 6 with the gradient, whose
// b2 enters as a float32 head and tail; per trigger term: 5.
//
// Work items: one compensator item per (request, row tile), then one pair item per (group,
// row tile, slice), the slice being an equal share of the union of the group's column
// windows (columns outside a request's own window add exact zeros for it). Row sums
// accumulate in float32 over the item's columns, then in float64 shared memory for the
// row tile's merge tree; the CTA completing a tree runs the epilogue of every request of its
// group (hk_internal.h). Results are deterministic for a given batch; they differ from the
// single-request kernel's only by float32 rounding (raw rather than scaled time differences,
// sums over an item rather than a tile).
#include "hk_internal.h"

#ifndef HK_GROUP_MIN_CTAS
#define HK_GROUP_MIN_CTAS 4  // resident CTAs per SM: 128 registers (7% faster than 3 CTAs at 164)
#endif

namespace hk {
namespace {

constexpr int kGThreads = kRowTile / 2;  // two rows (one packed pair) per thread
constexpr int kGWarpRows = 64;           // consecutive rows per warp
constexpr float kPadRaw = 1.0e18f;       // time of a padded event: dt^2 stays finite
static_assert(kGThreads <= 32 * kMaxCtaWarps, "CTA too wide");
// exact-zero gaps (scaled units, as in the single-request kernel)
constexpr float kGBgZero = 11.5157f;    // 1.01 * sqrt(130)
constexpr float kGTrigZero = 132.31f;   // 1.01 * 131

__device__ __forceinline__ float gex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int G, int NS>
struct GAcc {
  float2 v[G][NS];
};

template <int G>
struct GConst {
  float2 a2[G], b2[G], b2lo[G], cn[G], wn[G];
};

// One column tile against this thread's two rows for every request of the group. KIND as in
// the single-request kernel: 0 background only, 1 both terms with every pair causal, 2 both
// terms with the causal test (and the n' = n mask when excluding self), 3 trigger only. Every
// request of the group is evaluated (a request past its own exact-zero reach adds exact zeros):
// branch-free code over the group pays more than skipping does.
template <int KIND, int G, bool GRAD>
__device__ __forceinline__ void gtile_pass(const float4 *__restrict__ sxy, const float2 *__restrict__ st, float2 X,
                                           float2 Y, float2 T, int lo_a, int lo_b, int row_a, int c0, bool excl,
                                           const GConst<G> &K, GAcc<G, GRAD ? kSumsGrad : kSumsLoglik> &acc) {
  constexpr bool kBg = KIND != 3;
  constexpr bool kTrig = KIND != 0;
#pragma unroll 2
  for (int j = 0; j < kColTile; ++j) {
    const float4 c = sxy[j];  // {-x, -x, -y, -y}
    const float2 ct = st[j];  // {-t, -t}, the stored times
    const float2 dx = __fadd2_rn(X, make_float2(c.x, c.y));
    const float2 dy = __fadd2_rn(Y, make_float2(c.z, c.w));
    const float2 rho = __ffma2_rn(dy, dy, __fmul2_rn(dx, dx));
    const float2 dt = __fadd2_rn(T, ct);
    float2 u = make_float2(0.f, 0.f);
    if (kBg) u = __fmul2_rn(dt, dt);
    const int col = c0 + j;
#pragma unroll
    for (int k = 0; k < G; ++k) {
      {
        if (kBg) {
          // with the gradient, b2 enters as head + tail, so that u b2 is the correctly rounded
          // product with the float64 b2: a float32-rounded b2 would shift tau_t for every pair,
          // and d ell / d tau_t, nearly stationary on the N = 85,000 workload, would show it
          const float2 ub = GRAD ? __ffma2_rn(u, K.b2[k], __fmul2_rn(u, K.b2lo[k])) : __fmul2_rn(u, K.b2[k]);
          const float2 q = __ffma2_rn(rho, K.a2[k], ub);
          float2 eb = make_float2(gex2(-q.x), gex2(-q.y));
          if (KIND == 2 && excl) {
            if (col == row_a) eb.x = 0.f;
            if (col == row_a + 32) eb.y = 0.f;
          }
          acc.v[k][0] = __fadd2_rn(acc.v[k][0], eb);
          if (GRAD) {
            acc.v[k][2] = __ffma2_rn(rho, eb, acc.v[k][2]);
            acc.v[k][3] = __ffma2_rn(u, eb, acc.v[k][3]);
          }
        }
        if (kTrig) {
          const float2 arg = __ffma2_rn(rho, K.cn[k], __fmul2_rn(dt, K.wn[k]));
          float2 es = make_float2(gex2(arg.x), gex2(arg.y));
          if (KIND == 2) {
            es.x = col < lo_a ? es.x : 0.f;
            es.y = col < lo_b ? es.y : 0.f;
          }
          acc.v[k][1] = __fadd2_rn(acc.v[k][1], es);
          if (GRAD) {
            acc.v[k][4] = __ffma2_rn(rho, es, acc.v[k][4]);
            acc.v[k][5] = __ffma2_rn(dt, es, acc.v[k][5]);
          }
        }
      }
    }
  }
}

// A float32 row sum v >= 0 into a fixed-point accumulator as round(v 2^F) (scale = 2^F); a value
// that is not finite or reaches 2^62 is not added and sets the CTA's flag *bad.
__device__ __forceinline__ void gred_fix(long long *p, float v, float scale, int *bad) {
  const float x = v * scale;
  if (x == 0.f) return;
  if (!(fabsf(x) < 0x1p62f)) { *bad = 1; return; }
  atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)__float2ll_rn(x));
}

struct GStage {
  float4 sxy[2][kColTile];
  float2 st[2][kColTile];
};

__device__ __forceinline__ void gstage(const SetView &S, int ct, float4 *sxy, float2 *st) {
  for (int jj = threadIdx.x; jj < kColTile; jj += kGThreads) {
    const int j = ct * kColTile + jj;
    const float x = __ldg(S.x32 + j), y = __ldg(S.y32 + j);
    const float t = j < S.n ? __ldg(S.t32 + j) : kPadRaw;
    sxy[jj] = make_float4(-x, -x, -y, -y);
    st[jj] = make_float2(-t, -t);
  }
}

template <int G, bool GRAD>
__device__ void group_item(const Batch &B, int leader, int gsize, const PairItem &it, unsigned char *smem) {
  constexpr int NS = GRAD ? kSumsGrad : kSumsLoglik;
  const Request &R0 = B.req[leader];
  const SetView &S = R0.set;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rt = it.rt, row0 = rt * kRowTile, n = S.n;
  const int wa = row0 + warp * kGWarpRows, wb = wa + kGWarpRows - 1;
  const int lo_wa = S.lo32[wa], lo_wb = S.lo32[wb];
  const bool excl = (R0.flags & kFlagExcludeSelf) != 0;
  const int ra = wa + lane, rb = ra + 32;
  const float2 X = make_float2(S.x32[ra], S.x32[rb]);
  const float2 Y = make_float2(S.y32[ra], S.y32[rb]);
  const float2 T = make_float2(ra < n ? S.t32[ra] : kPadRaw, rb < n ? S.t32[rb] : kPadRaw);
  const int lo_a = S.lo32[ra], lo_b = S.lo32[rb];

  // per-request constants, the group's column window (union) and its exact-zero gaps (days)
  GConst<G> K;
  int c_lo = S.nct, c_hi = 0;
  float bg_gap = 0.f, trig_gap = 0.f;  // the group's largest exact-zero gaps (days)
  const double log2e = 1.4426950408889634074;
#pragma unroll
  for (int k = 0; k < G; ++k) {
    const Request &R = B.req[leader + (k < gsize ? k : 0)];
    const float b2 = R.b2;
    K.a2[k] = make_float2(R.a2, R.a2);
    K.b2[k] = make_float2(b2, b2);
    K.b2lo[k] = make_float2(R.b2_lo, R.b2_lo);
    K.cn[k] = make_float2(R.cn, R.cn);
    const float wn = (float)(-R.omega * log2e);
    K.wn[k] = make_float2(wn, wn);
    if (k < gsize) {
      const int2 w = table_window_rt(R, S.win32, S.t32, rt);
      if (w.x >= 0) {
        c_lo = min(c_lo, w.x);
        c_hi = max(c_hi, w.y);
      } else {
        c_lo = 0;
        c_hi = S.nct;
      }
      bg_gap = fmaxf(bg_gap, kGBgZero / R.beta);
      trig_gap = fmaxf(trig_gap, (float)(kGTrigZero / (R.omega * log2e)));
    }
  }
  const int width = c_hi - c_lo;
  const int ns = R0.slices, l0 = it.node * it.span, l1 = min(l0 + it.span, ns);
  const int c_begin = c_lo + (int)((long long)width * l0 / ns), c_end = c_lo + (int)((long long)width * l1 / ns);

  GStage &sg = *reinterpret_cast<GStage *>(smem);
  GAcc<G, NS> acc;
#pragma unroll
  for (int k = 0; k < G; ++k)
#pragma unroll
    for (int s = 0; s < NS; ++s) acc.v[k][s] = make_float2(0.f, 0.f);
  const float t_first = __shfl_sync(0xffffffffu, T.x, 0);  // the warp's first and last rows
  const float t_last = __shfl_sync(0xffffffffu, T.y, 31);
  if (c_begin < c_end) {
    gstage(S, c_begin, sg.sxy[0], sg.st[0]);
    __syncthreads();
  }
  for (int ct = c_begin, k = 0; ct < c_end; ++ct, ++k) {
    const int buf = k & 1;
    const int c0 = ct * kColTile, c1 = c0 + kColTile;
    int kind;  // for the group as a whole (largest reaches)
    if (c1 <= lo_wa) {  // every pair causal
      const float gap = t_first + sg.st[buf][kColTile - 1].x;  // first row - latest column
      const bool bg_zero = gap >= bg_gap, trig_zero = gap >= trig_gap;
      kind = bg_zero ? (trig_zero ? -1 : 3) : (trig_zero ? 0 : 1);
    } else if (c0 >= lo_wb) {  // no causal pair
      const float gap = -sg.st[buf][0].x - t_last;  // earliest column - last row
      kind = gap >= bg_gap ? -1 : 0;
    } else {
      kind = 2;
    }
    if (excl && c0 <= wb && c1 > wa) kind = 2;
    if (kind == 0)
      gtile_pass<0, G, GRAD>(sg.sxy[buf], sg.st[buf], X, Y, T, lo_a, lo_b, ra, c0, excl, K, acc);
    else if (kind == 1)
      gtile_pass<1, G, GRAD>(sg.sxy[buf], sg.st[buf], X, Y, T, lo_a, lo_b, ra, c0, excl, K, acc);
    else if (kind == 2)
      gtile_pass<2, G, GRAD>(sg.sxy[buf], sg.st[buf], X, Y, T, lo_a, lo_b, ra, c0, excl, K, acc);
    else if (kind == 3)
      gtile_pass<3, G, GRAD>(sg.sxy[buf], sg.st[buf], X, Y, T, lo_a, lo_b, ra, c0, excl, K, acc);
    if (ct + 1 < c_end) gstage(S, ct + 1, sg.sxy[buf ^ 1], sg.st[buf ^ 1]);
    __syncthreads();
  }

  const int la = warp * kGWarpRows + lane, lb = la + 32;
  if (R0.fixsum) {
    // Fixed-point sums (every request of the batch has them, see Request::fixsum): each
    // request's row sums go to its own per-event integers, round(v 2^F) with the request's
    // scales, then the item arrives at its row tile's counter (the leader's rt_done); the item
    // that completes the row tile runs the epilogue of every request of the group.
    __shared__ int s_bad;
    __shared__ unsigned s_last;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    const size_t np = (size_t)S.npad;
#pragma unroll
    for (int k = 0; k < G; ++k) {
      if (k >= gsize) break;
      const Request &R = B.req[leader + k];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const float scale = __int_as_float((127 + R.fix_bits[s]) << 23);
        gred_fix(R.fixsum + s * np + row0 + la, acc.v[k][s].x, scale, &s_bad);
        gred_fix(R.fixsum + s * np + row0 + lb, acc.v[k][s].y, scale, &s_bad);
      }
    }
    __syncthreads();
    if (tid == 0 && s_bad)
      for (int k = 0; k < gsize; ++k)
        if (B.req[leader + k].status) atomicOr(B.req[leader + k].status, kStatusFixRange);
    __threadfence();
    __syncthreads();
    const unsigned items = (unsigned)rowtile_items(R0, it.span);
    const unsigned add = it.node == 0 ? kSymRootMark - (items - 1u) : 1u;
    if (tid == 0) s_last = atomicAdd(R0.rt_done + rt, add) + add == kSymRootMark;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int k = 0; k < gsize; ++k) {
      const Request &R = B.req[leader + k];
      double v[GRAD ? 7 : 1] = {};
      const int rows[2] = {la, lb};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = row0 + rows[h];
        if (i < n) {
          double sums[NS];
#pragma unroll
          for (int s = 0; s < NS; ++s)
            sums[s] = (double)__ldcg(R.fixsum + s * np + i) * __longlong_as_double((long long)(1023 - R.fix_bits[s]) << 52);
          row_terms<GRAD>(R, B.mix2, i, sums, v);
        }
      }
      rowtile_reduce<GRAD>(R, B.mix2, rt, v);
    }
    return;
  }
  // float64 sums of the group's requests for this thread's rows; they reuse the staging space
  double *gsum = reinterpret_cast<double *>(smem);  // [G][NS][kRowTile]
#pragma unroll
  for (int k = 0; k < G; ++k)
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      gsum[(k * NS + s) * kRowTile + la] = (double)acc.v[k][s].x;
      gsum[(k * NS + s) * kRowTile + lb] = (double)acc.v[k][s].y;
    }
  auto store = [&](int to) {
    for (int k = 0; k < gsize; ++k) {
      double *dst = B.req[leader + k].partials + (size_t)to * NS * kRowTile;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        dst[s * kRowTile + la] = gsum[(k * NS + s) * kRowTile + la];
        dst[s * kRowTile + lb] = gsum[(k * NS + s) * kRowTile + lb];
      }
    }
  };
  if (!B.fused) {  // row-tile-major slot of the item's first leaf (unfused launches use 1-leaf items)
    store(rt * ns + l0);
    return;
  }
  auto merge = [&](int from) {
    for (int k = 0; k < gsize; ++k) {
      const double *src = B.req[leader + k].partials + (size_t)from * NS * kRowTile;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        gsum[(k * NS + s) * kRowTile + la] += __ldcg(src + s * kRowTile + la);
        gsum[(k * NS + s) * kRowTile + lb] += __ldcg(src + s * kRowTile + lb);
      }
    }
  };
  const int root = merge_tree<GRAD>(R0, it, store, merge);
  if (root < 0)
    for (int k = 0; k < gsize; ++k) mark_timeout(B.req[leader + k]);
  if (root <= 0) return;
  for (int k = 0; k < gsize; ++k) {
    const Request &R = B.req[leader + k];
    double v[GRAD ? 7 : 1] = {};
    const int rows[2] = {la, lb};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = row0 + rows[h];
      if (i < n) {
        double sums[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) sums[s] = gsum[(k * NS + s) * kRowTile + rows[h]];
        row_terms<GRAD>(R, B.mix2, i, sums, v);
      }
    }
    rowtile_reduce<GRAD>(R, B.mix2, rt, v);
  }
}

template <int G, bool GRAD>
__global__ void __launch_bounds__(kGThreads, HK_GROUP_MIN_CTAS) pair_group_kernel(const __grid_constant__ Batch B) {
  extern __shared__ __align__(16) unsigned char gsmem[];
  const int item = blockIdx.x;
  const int nrt = B.req[0].set.nrt;
  if (item < B.comp_total) {  // compensator item of (request item / nrt, row tile item % nrt)
    const Request &R = B.req[item / nrt];
    compensator_tile(R, B.mix2, R.set.t32, item % nrt, GRAD);
    if (B.fused) finish_request<GRAD>(R);
    return;
  }
  const int per_group = pair_items(B.req[0]);
  const int p = item - B.comp_total, g = p / per_group, local = p - g * per_group;
  const int leader = g * G, gsize = min(G, B.nreq - leader);
  group_item<G, GRAD>(B, leader, gsize, item_at(B.req[leader], local), gsmem);
}

template <int G, bool GRAD>
cudaError_t launch_group(const Batch &b, cudaStream_t s) {
  constexpr size_t sums = (size_t)G * (GRAD ? kSumsGrad : kSumsLoglik) * kRowTile * sizeof(double);
  constexpr size_t smem = sums > sizeof(GStage) ? sums : sizeof(GStage);
  cudaError_t e = cudaFuncSetAttribute(pair_group_kernel<G, GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  pair_group_kernel<G, GRAD><<<b.total_items, kGThreads, smem, s>>>(b);
  return cudaGetLastError();
}

}  // namespace

static_assert(sizeof(kGroupSizesGrad) == sizeof(int) && kGroupSizesGrad[0] == 4,
              "the launcher below instantiates these group sizes");
static_assert(sizeof(kGroupSizesLoglik) == 2 * sizeof(int) && kGroupSizesLoglik[0] == 4 && kGroupSizesLoglik[1] == 8,
              "the launcher below instantiates these group sizes");

cudaError_t launch_pair_group(const Batch &b, bool grad, cudaStream_t s) {
  if (b.total_items < 1) return cudaErrorInvalidValue;
  if (grad && b.group == 4) return launch_group<4, true>(b, s);
  if (!grad && b.group == 4) return launch_group<4, false>(b, s);
  if (!grad && b.group == 8) return launch_group<8, false>(b, s);
  return cudaErrorInvalidValue;
}

}  // namespace hk
