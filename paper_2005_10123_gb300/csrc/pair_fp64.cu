// Double-precision pair kernel.
//
// pair_fp64_kernel forms the same per-row sums as the mixed kernel (S_b, S_s and the
// gradient moments R_b, T_b, R_s, U_s of Section 2.1, Eq. 1), entirely in float64 with
// the library exp(), and the moments in raw units (r^2 in km^2, dt in days). Compensator
// items sum each row tile's compensator terms, and the CTA that completes a row tile's merge
// tree runs its fused epilogue (hk_internal.h: merge_tree, row_terms, rowtile_reduce).
#include "hk_internal.h"

namespace hk {
namespace {

#ifndef HK_FP64_MIN_CTAS
#define HK_FP64_MIN_CTAS 1  // resident CTAs per SM the register budget must allow
#endif

constexpr double kPadTime = 1.0e150;  // time of a padded event: dt^2 = 1e300 stays finite
// Each thread holds 4 rows; a CTA covers the row tile with kRowTile / 4 threads and each
// warp owns 128 consecutive rows.
constexpr int kRows64 = 4;
constexpr int kThreads64 = kRowTile / kRows64;
constexpr int kWarpRows64 = 32 * kRows64;
// Slices cut the column window at kChunk64-column granularity (float64 pair work is slow
// enough that a small set needs items smaller than a column tile to fill the GPU).
#ifndef HK_CHUNK64
#define HK_CHUNK64 8  // N = 2,000 loglik: 0.43 ms with 32-column chunks, 0.36 with 8
#endif
constexpr int kChunk64 = HK_CHUNK64;
constexpr int kChunksPerTile64 = kColTile / kChunk64;
static_assert(kColTile % kChunk64 == 0, "column chunks must tile a column tile");

// With a two-component trigger mixture (MIX = 2) component 2 (omega2, dc2) goes to the sums after
// the single-kernel ones.
template <int KIND, bool GRAD, int MIX>
__device__ __forceinline__ void tile_pass64(const double *__restrict__ sx, const double *__restrict__ sy,
                                            const double *__restrict__ st, const double (&X)[4],
                                            const double (&Y)[4], const double (&T)[4], const int (&LO)[4],
                                            int row_a0, int c0, int j0, int j1, bool excl, double da, double db,
                                            double dc, double omega, double dc2, double omega2,
                                            double (&acc)[num_sums(GRAD, MIX)][4]) {
  constexpr int S2 = GRAD ? 6 : 2;
#pragma unroll 2
  for (int j = j0; j < j1; ++j) {
    const double cx = sx[j], cy = sy[j], ctj = st[j];
    const int col = c0 + j;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double dx = X[k] - cx, dy = Y[k] - cy, dt = T[k] - ctj;
      const double r2 = __fma_rn(dx, dx, __dmul_rn(dy, dy));
      if (KIND != 3) {  // KIND 3: every background term of the tile is exactly zero
        const double u = __dmul_rn(dt, dt);
        double eb = exp(-__fma_rn(r2, da, __dmul_rn(u, db)));
        if (KIND == 2 && excl && col == row_a0 + 32 * k) eb = 0.0;
        acc[0][k] += eb;
        if (GRAD) {
          acc[2][k] = __fma_rn(r2, eb, acc[2][k]);
          acc[3][k] = __fma_rn(u, eb, acc[3][k]);
        }
      }
      if (KIND != 0) {
        double es = exp(-__fma_rn(omega, dt, __dmul_rn(r2, dc)));
        if (KIND == 2) es = (col < LO[k]) ? es : 0.0;
        acc[1][k] += es;
        if (GRAD) {
          acc[4][k] = __fma_rn(r2, es, acc[4][k]);
          acc[5][k] = __fma_rn(dt, es, acc[5][k]);
        }
        if (MIX > 1) {
          double es2 = exp(-__fma_rn(omega2, dt, __dmul_rn(r2, dc2)));
          if (KIND == 2) es2 = (col < LO[k]) ? es2 : 0.0;
          acc[S2][k] += es2;
          if (GRAD) {
            acc[S2 + 1][k] = __fma_rn(r2, es2, acc[S2 + 1][k]);
            acc[S2 + 2][k] = __fma_rn(dt, es2, acc[S2 + 2][k]);
          }
        }
      }
    }
  }
}

template <bool GRAD, int MIX>
__device__ void run_piece64(const Batch &B, const Request &R, const PairItem &it, int4 piece, double (*sx)[kColTile],
                            double (*sy)[kColTile], double (*st)[kColTile]) {
  constexpr int NS = num_sums(GRAD, MIX);
  const SetView &S = R.set;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int row0 = piece.x * kRowTile;
  const int n = S.n;
  const int wa = row0 + warp * kWarpRows64, wb = wa + kWarpRows64 - 1;
  const int lo_wa = S.lo64[wa], lo_wb = S.lo64[wb];
  const bool excl = (R.flags & 1) != 0;
  const double da = R.da, db = R.db, dc = R.dc, omega = R.omega;
  const double dc2 = B.mix2.dc2, omega2 = B.mix2.omega2;
  // gaps (days) between the warp's earliest row and a tile's latest column past which every
  // background (bg_gap) or trigger (trig_gap) term of the tile contributes nothing at float64
  // precision: the host's reaches with their one percent of margin (term_reaches in api.cu)
  const double bg_gap = R.cut_late, trig_gap = R.trig_cut;

  double X[4], Y[4], T[4];
  int LO[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = wa + lane + 32 * k;
    X[k] = S.x64[r];
    Y[k] = S.y64[r];
    T[k] = r < n ? S.t64[r] : kPadTime;
    LO[k] = S.lo64[r];
  }
  const double t_first = __shfl_sync(0xffffffffu, T[0], 0);  // the warp's earliest row
  const double t_last = __shfl_sync(0xffffffffu, T[3], 31);  // and its latest (padding: +huge)
  double acc[NS][4];
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[s][k] = 0.0;

  auto stage = [&](int ct, int buf) {
    for (int jj = threadIdx.x; jj < kColTile; jj += kThreads64) {
      const int j = ct * kColTile + jj;
      sx[buf][jj] = S.x64[j];
      sy[buf][jj] = S.y64[j];
      st[buf][jj] = j < n ? S.t64[j] : kPadTime;
    }
  };
  // piece.y, piece.z: the item's column range in kChunk64-column chunks
  const int col_begin = piece.y * kChunk64, col_end = piece.z * kChunk64;
  int ct = piece.y / kChunksPerTile64;
  const int ct_end = piece.y < piece.z ? (piece.z - 1) / kChunksPerTile64 + 1 : ct;
  if (ct < ct_end) {  // an empty slice of the window writes zero partial sums
    stage(ct, 0);
    __syncthreads();
  }
  for (int k = 0; ct < ct_end; ++ct, ++k) {
    const int buf = k & 1;
    const int c0 = ct * kColTile, c1 = c0 + kColTile;
    const int j0 = max(col_begin - c0, 0), j1 = min(col_end - c0, kColTile);
    int kind;
    if (c1 <= lo_wa) {  // every pair causal: which of the two terms can be nonzero?
      const double gap = t_first - st[buf][kColTile - 1];
      const bool bg_zero = gap >= bg_gap, trig_zero = gap >= trig_gap;
      kind = bg_zero ? (trig_zero ? -1 : 3) : (trig_zero ? 0 : 1);
    } else if (c0 >= lo_wb) {  // no causal pair: background only, zero past its reach
      kind = st[buf][0] - t_last >= bg_gap ? -1 : 0;
    } else {
      kind = 2;
    }
    if (excl && c0 <= wb && c1 > wa) kind = 2;
    const int row_a0 = wa + lane;
    if (kind == 0)
      tile_pass64<0, GRAD, MIX>(sx[buf], sy[buf], st[buf], X, Y, T, LO, row_a0, c0, j0, j1, excl, da, db, dc, omega,
                                dc2, omega2, acc);
    else if (kind == 1)
      tile_pass64<1, GRAD, MIX>(sx[buf], sy[buf], st[buf], X, Y, T, LO, row_a0, c0, j0, j1, excl, da, db, dc, omega,
                                dc2, omega2, acc);
    else if (kind == 2)
      tile_pass64<2, GRAD, MIX>(sx[buf], sy[buf], st[buf], X, Y, T, LO, row_a0, c0, j0, j1, excl, da, db, dc, omega,
                                dc2, omega2, acc);
    else if (kind == 3)
      tile_pass64<3, GRAD, MIX>(sx[buf], sy[buf], st[buf], X, Y, T, LO, row_a0, c0, j0, j1, excl, da, db, dc, omega,
                                dc2, omega2, acc);
    if (ct + 1 < ct_end) stage(ct + 1, buf ^ 1);
    __syncthreads();
  }
  // this thread's rows: li = warp * kWarpRows64 + lane + 32 k, sums in acc[s][k]
  auto store = [&](int to) {
    double *dst = R.partials + (size_t)to * NS * kRowTile;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int s = 0; s < NS; ++s) dst[s * kRowTile + warp * kWarpRows64 + lane + 32 * k] = acc[s][k];
  };
  if (!B.fused) {  // row-tile-major slot of the item's first leaf (unfused launches use 1-leaf items)
    store(it.rt * R.slices + it.node * it.span);
    return;
  }
  auto merge = [&](int from) {
    const double *src = R.partials + (size_t)from * NS * kRowTile;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int s = 0; s < NS; ++s) acc[s][k] += __ldcg(src + s * kRowTile + warp * kWarpRows64 + lane + 32 * k);
  };
  const int root = merge_tree<true>(R, it, store, merge);
  if (root < 0) mark_timeout(R);
  if (root <= 0) return;
  double v[GRAD ? 1 + NS : 1] = {};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = row0 + warp * kWarpRows64 + lane + 32 * k;
    if (i < n) {
      double sums[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) sums[s] = acc[s][k];
      row_terms<GRAD, MIX>(R, B.mix2, i, sums, v);
    }
  }
  rowtile_reduce<GRAD, MIX>(R, B.mix2, piece.x, v);
}

template <bool GRAD, int MIX>
__global__ void __launch_bounds__(kThreads64, HK_FP64_MIN_CTAS) pair_fp64_kernel(const __grid_constant__ Batch B) {
  __shared__ double sx[2][kColTile], sy[2][kColTile], st[2][kColTile];
  __shared__ int2 s_win;
  const int item = blockIdx.x;
  const Request &R = B.req[find_request(B, item)];
  const int local = item - R.item_begin, nc = comp_items(R);
  if (local < nc) {  // compensator item of row tile `local`
    compensator_tile<MIX>(R, B.mix2, R.set.t64, local, GRAD);
    if (B.fused) finish_request<GRAD, MIX>(R);
    return;
  }
  const PairItem it = item_at(R, local - nc);
  const int rt = it.rt, ns = R.slices, l0 = it.node * it.span, l1 = min(l0 + it.span, ns);
  int2 w = table_window_rt(R, R.set.win64, R.set.t64, rt);
  if (w.x < 0) {  // no lookup table: one warp searches the times
    if (threadIdx.x < 32) {
      const int2 v = column_window(R, R.set.t64, rt);
      if (threadIdx.x == 0) s_win = v;
    }
    __syncthreads();
    w = s_win;
  }
  // the window in column chunks, cut into `ns` near-equal leaves
  const int cw0 = w.x * kChunksPerTile64, width = (w.y - w.x) * kChunksPerTile64;
  const int c_begin = cw0 + (int)((long long)width * l0 / ns);
  const int c_end = cw0 + (int)((long long)width * l1 / ns);
  run_piece64<GRAD, MIX>(B, R, it, make_int4(rt, c_begin, c_end, 0), sx, sy, st);
}

}  // namespace

cudaError_t launch_pair_fp64(const Batch &b, bool grad, cudaStream_t s) {
  if (b.total_items < 1) return cudaErrorInvalidValue;
  if (b.req[0].mix > 1) {  // a trigger mixture (one request per launch)
    if (grad) pair_fp64_kernel<true, 2><<<b.total_items, kThreads64, 0, s>>>(b);
    else pair_fp64_kernel<false, 2><<<b.total_items, kThreads64, 0, s>>>(b);
  } else if (grad) {
    pair_fp64_kernel<true, 1><<<b.total_items, kThreads64, 0, s>>>(b);
  } else {
    pair_fp64_kernel<false, 1><<<b.total_items, kThreads64, 0, s>>>(b);
  }
  return cudaGetLastError();
}

int fp64_chunks_per_tile() { return kChunksPerTile64; }

int occupancy_pair_fp64(bool grad) {
  int n = 0;
  if (grad) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_fp64_kernel<true, 1>, kThreads64, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_fp64_kernel<false, 1>, kThreads64, 0);
  return n;
}

}  // namespace hk
