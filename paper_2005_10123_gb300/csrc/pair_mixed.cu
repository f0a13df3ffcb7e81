// Mixed-precision pair kernel: float32 pair terms, float32 accumulation over one
// 256-column tile, float64 accumulation across tiles.
//
// For every row (event n) of its row tile the kernel forms, over the columns n' of
// its work range (Section 2.1, Eq. 1 inner sum; gradient moments added here):
//   S_b = sum_n'          e_b,  e_b = exp(-r^2/(2 tau_x^2) - dt^2/(2 tau_t^2))
//   S_s = sum_{t_n' < t_n} e_s,  e_s = exp(-omega dt - r^2/(2 h^2))
//   R_b = sum r^2 e_b,  T_b = sum dt'^2 e_b,  R_s = sum r^2 e_s,  U_s = sum dt' e_s
// with r^2 = |x_n - x_n'|^2, dt = t_n - t_n' and dt' = beta dt (beta^2 = log2(e)/(2 tau_t^2)).
// The epilogue kernel turns the row sums into lambda_n, log lambda_n and the gradient.
//
// Arithmetic per (row, column) pair, two rows per packed f32x2 instruction:
//   dx, dy exact differences of the stored float32 coordinates; r^2 = dx^2 + dy^2;
//   dt' = T_n - t'_n' where both times are taken relative to the first row of the
//   tile before scaling, so nearby times keep full relative precision;
//   e_b = 2^-(a2 r^2 + dt'^2),  e_s = 2^(cn r^2 + wn dt')  (ex2.approx.ftz).
// The causal indicator t_n' < t_n is tested on stored times through lo[n] (the first
// index whose stored time equals t_n): for sorted times, t_n' < t_n  <=>  n' < lo[n].
// Column tiles entirely before a warp's rows skip the test, tiles entirely after skip
// the trigger term; only tiles straddling the rows test pair by pair.
#include "hk_internal.h"

namespace hk {
namespace {

constexpr float kPadScaled = 1.0e18f;  // scaled time of a padded event: dt'^2 = 1e36 stays finite

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int NS>
struct Acc32 {
  float2 v[NS][kRowsPerThread / 2];
};

// One column tile against this thread's rows. KIND 0: no causal pair in the tile for
// this warp; 1: every pair causal; 2: test each pair (and mask n' = n if excluding self).
template <int KIND, bool GRAD>
__device__ __forceinline__ void tile_pass(const float4 *__restrict__ sxy, const float2 *__restrict__ st,
                                          const float2 (&X)[2], const float2 (&Y)[2], const float2 (&T)[2],
                                          const int (&LO)[4], int row_a0, int c0, bool excl, float2 A2,
                                          float2 WN, float2 CN, Acc32<GRAD ? kSumsGrad : kSumsLoglik> &acc) {
#pragma unroll 4
  for (int j = 0; j < kColTile; ++j) {
    const float4 c = sxy[j];   // {-x, -x, -y, -y}
    const float2 ctn = st[j];  // {-t', -t'}
    const float2 cx = make_float2(c.x, c.y), cy = make_float2(c.z, c.w);
    const int col = c0 + j;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const float2 dx = __fadd2_rn(X[p], cx);
      const float2 dy = __fadd2_rn(Y[p], cy);
      float2 rho = __fmul2_rn(dx, dx);
      rho = __ffma2_rn(dy, dy, rho);
      const float2 dt = __fadd2_rn(T[p], ctn);
      const float2 u = __fmul2_rn(dt, dt);
      const float2 q = __ffma2_rn(rho, A2, u);
      float2 eb = make_float2(ex2(-q.x), ex2(-q.y));
      if (KIND == 2 && excl) {
        const int ra = row_a0 + 64 * p;
        if (col == ra) eb.x = 0.f;
        if (col == ra + 32) eb.y = 0.f;
      }
      acc.v[0][p] = __fadd2_rn(acc.v[0][p], eb);
      if (GRAD) {
        acc.v[2][p] = __ffma2_rn(rho, eb, acc.v[2][p]);
        acc.v[3][p] = __ffma2_rn(u, eb, acc.v[3][p]);
      }
      if (KIND != 0) {
        const float2 v = __fmul2_rn(dt, WN);
        const float2 arg = __ffma2_rn(rho, CN, v);
        float2 es = make_float2(ex2(arg.x), ex2(arg.y));
        if (KIND == 2) {
          es.x = (col < LO[2 * p]) ? es.x : 0.f;
          es.y = (col < LO[2 * p + 1]) ? es.y : 0.f;
        }
        acc.v[1][p] = __fadd2_rn(acc.v[1][p], es);
        if (GRAD) {
          acc.v[4][p] = __ffma2_rn(rho, es, acc.v[4][p]);
          acc.v[5][p] = __ffma2_rn(dt, es, acc.v[5][p]);
        }
      }
    }
  }
}

struct RawCols {
  float x0, y0, t0, x1, y1, t1;
};

__device__ __forceinline__ RawCols load_cols(const SetView &S, int ct, int tid) {
  const int j0 = ct * kColTile + tid, j1 = j0 + kThreads;
  RawCols r;
  r.x0 = __ldg(S.x32 + j0); r.y0 = __ldg(S.y32 + j0); r.t0 = __ldg(S.t32 + j0);
  r.x1 = __ldg(S.x32 + j1); r.y1 = __ldg(S.y32 + j1); r.t1 = __ldg(S.t32 + j1);
  return r;
}

__device__ __forceinline__ void store_cols(const RawCols &r, int ct, int tid, int n, float t_origin,
                                           float beta, float4 *sxy, float2 *st) {
  const int j0 = ct * kColTile + tid, j1 = j0 + kThreads;
  const float s0 = j0 < n ? (r.t0 - t_origin) * beta : kPadScaled;
  const float s1 = j1 < n ? (r.t1 - t_origin) * beta : kPadScaled;
  sxy[tid] = make_float4(-r.x0, -r.x0, -r.y0, -r.y0);
  st[tid] = make_float2(-s0, -s0);
  sxy[tid + kThreads] = make_float4(-r.x1, -r.x1, -r.y1, -r.y1);
  st[tid + kThreads] = make_float2(-s1, -s1);
}

template <bool GRAD>
__device__ void run_piece(const Request &R, int4 piece, int slot, float4 (*sxy)[kColTile],
                          float2 (*st)[kColTile]) {
  constexpr int NS = GRAD ? kSumsGrad : kSumsLoglik;
  const SetView &S = R.set;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int row0 = piece.x * kRowTile;
  const float t_origin = S.t32[row0];
  const float beta = R.beta;
  const int n = S.n;
  const int wa = row0 + warp * kWarpRows, wb = wa + kWarpRows - 1;
  const int lo_wa = S.lo32[wa], lo_wb = S.lo32[wb];
  const bool excl = (R.flags & 1) != 0;

  float2 X[2], Y[2], T[2];
  int LO[4];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int ra = wa + lane + 64 * p, rb = ra + 32;
    X[p] = make_float2(S.x32[ra], S.x32[rb]);
    Y[p] = make_float2(S.y32[ra], S.y32[rb]);
    T[p] = make_float2(ra < n ? (S.t32[ra] - t_origin) * beta : kPadScaled,
                       rb < n ? (S.t32[rb] - t_origin) * beta : kPadScaled);
    LO[2 * p] = S.lo32[ra];
    LO[2 * p + 1] = S.lo32[rb];
  }
  const float2 A2 = make_float2(R.a2, R.a2), WN = make_float2(R.wn, R.wn), CN = make_float2(R.cn, R.cn);

  double acc64[NS][kRowsPerThread];
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) acc64[s][k] = 0.0;

  int ct = piece.y;
  store_cols(load_cols(S, ct, tid), ct, tid, n, t_origin, beta, sxy[0], st[0]);
  __syncthreads();
  for (int k = 0; ct < piece.z; ++ct, ++k) {
    const int buf = k & 1;
    const bool has_next = ct + 1 < piece.z;
    RawCols nxt;
    if (has_next) nxt = load_cols(S, ct + 1, tid);
    const int c0 = ct * kColTile, c1 = c0 + kColTile;
    int kind = (c1 <= lo_wa) ? 1 : (c0 >= lo_wb ? 0 : 2);
    if (excl && c0 <= wb && c1 > wa) kind = 2;
    Acc32<NS> acc;
#pragma unroll
    for (int s = 0; s < NS; ++s) acc.v[s][0] = acc.v[s][1] = make_float2(0.f, 0.f);
    const int row_a0 = wa + lane;
    if (kind == 0)
      tile_pass<0, GRAD>(sxy[buf], st[buf], X, Y, T, LO, row_a0, c0, excl, A2, WN, CN, acc);
    else if (kind == 1)
      tile_pass<1, GRAD>(sxy[buf], st[buf], X, Y, T, LO, row_a0, c0, excl, A2, WN, CN, acc);
    else
      tile_pass<2, GRAD>(sxy[buf], st[buf], X, Y, T, LO, row_a0, c0, excl, A2, WN, CN, acc);
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        acc64[s][2 * p] += (double)acc.v[s][p].x;
        acc64[s][2 * p + 1] += (double)acc.v[s][p].y;
      }
    if (has_next) store_cols(nxt, ct + 1, tid, n, t_origin, beta, sxy[buf ^ 1], st[buf ^ 1]);
    __syncthreads();
  }
  double *dst = R.partials + (size_t)slot * NS * kRowTile;
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int la = warp * kWarpRows + lane + 64 * p;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      dst[s * kRowTile + la] = acc64[s][2 * p];
      dst[s * kRowTile + la + 32] = acc64[s][2 * p + 1];
    }
  }
}

template <bool GRAD>
__global__ void __launch_bounds__(kThreads, 4) pair_mixed_kernel(const __grid_constant__ Batch B) {
  __shared__ __align__(16) float4 sxy[2][kColTile];
  __shared__ __align__(16) float2 st[2][kColTile];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(B.counter, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= B.total_items) break;
    const Request &R = B.req[find_request(B, item, false)];
    const int range = item - R.item_begin;
    const int p0 = R.sched.range_first[range], p1 = R.sched.range_first[range + 1];
    for (int pc = p0; pc < p1; ++pc) run_piece<GRAD>(R, R.sched.pieces[pc], pc, sxy, st);
  }
}

}  // namespace

cudaError_t launch_pair_mixed(const Batch &b, bool grad, int grid, cudaStream_t s) {
  if (grad) pair_mixed_kernel<true><<<grid, kThreads, 0, s>>>(b);
  else pair_mixed_kernel<false><<<grid, kThreads, 0, s>>>(b);
  return cudaGetLastError();
}

int occupancy_pair_mixed(bool grad) {
  int n = 0;
  if (grad) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_mixed_kernel<true>, kThreads, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_mixed_kernel<false>, kThreads, 0);
  return n;
}

}  // namespace hk
