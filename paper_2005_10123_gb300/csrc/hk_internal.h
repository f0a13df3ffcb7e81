// Internal declarations shared by the kernels and the host runtime of the library.
// Not part of the public ABI (include/hawkes.h is).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hk {

// ---- tiling -------------------------------------------------------------------------
// A pair-kernel CTA holds kRowTile consecutive rows (events n) in registers,
// kRowsPerThread per thread, and streams column tiles of kColTile events (n')
// through shared memory. Event arrays are padded to a multiple of both tile sizes.
#ifndef HK_ROWS_PER_THREAD
#define HK_ROWS_PER_THREAD 4
#endif
#ifndef HK_THREADS
#define HK_THREADS 128
#endif
#ifndef HK_COL_TILE
#define HK_COL_TILE 256
#endif
constexpr int kThreads = HK_THREADS;
constexpr int kRowsPerThread = HK_ROWS_PER_THREAD;  // even: rows are processed in packed pairs
constexpr int kRowTile = kThreads * kRowsPerThread;  // 512 with 4 rows per thread
constexpr int kColTile = HK_COL_TILE;
constexpr int kWarpRows = 32 * kRowsPerThread;       // consecutive rows per warp
constexpr int kPadTo = kRowTile > kColTile ? kRowTile : kColTile;  // event arrays padded to this
constexpr int kEpiThreads = 256;                     // rows per CTA of the allocation-free epilogue
constexpr int kMaxBatch = 64;                        // requests per launch
constexpr int kSumsLoglik = 2;                       // S_b, S_s
constexpr int kSumsGrad = 6;                         // S_b, S_s, R_b, T_b, R_s, U_s
constexpr int kFlagExcludeSelf = 1;                  // HAWKES_FLAG_EXCLUDE_SELF
constexpr int kFlagDense = 2;                        // HAWKES_FLAG_DENSE
constexpr int kMaxCtaWarps = 8;                      // pair-kernel CTAs have at most 256 threads
static_assert(kThreads <= 32 * kMaxCtaWarps && kRowTile / 4 <= 32 * kMaxCtaWarps, "CTA too wide");

// One resident event set, as the kernels see it.
struct SetView {
  const float *x32, *y32, *t32;
  const double *x64, *y64, *t64;
  const int *lo32, *lo64;  // lo[i] = first index with the same stored time as event i
  int n, npad, nrt, nct;   // events, padded length, row tiles, column tiles
};

// Work decomposition: item = (row tile rt, slice s), s < slices. For each request the
// pair kernel finds the window of column tiles of rt that can hold a nonzero pair term
// (every other pair term is exactly zero at the working precision, see cut_early and
// cut_late) and gives slice s the s-th of `slices` near-equal parts of that window. The
// item index rt * slices + s is also the partial-sum slot, so results do not depend on
// which CTA ran which item.
struct Request {
  SetView set;
  int slices;      // slices per row tile (fixed per set and kernel kind)
  int grad;        // 0: loglik only; 1: loglik and gradient
  int flags;       // HAWKES_FLAG_* of the context at submission
  int item_begin;  // first pair-kernel item of this request in the batch
  // Column window: column n' can only contribute to row n if
  //   t_n - cut_early <= t_n' <= t_n + cut_late   (days; +inf keeps every column)
  double cut_early, cut_late;
  // float32 pair constants (mixed mode)
  float a2;    // log2(e) / (2 tau_x^2)                  multiplies r^2
  float beta;  // sqrt(log2(e) / (2 tau_t^2))            scales (t - t0)
  float wn;    // -omega log2(e) / beta                  multiplies scaled dt
  float cn;    // -log2(e) / (2 h^2)                     multiplies r^2
  // float64 pair constants (fp64 mode)
  double da;   // 1 / (2 tau_x^2)
  double db;   // 1 / (2 tau_t^2)
  double dc;   // 1 / (2 h^2)
  // Theta and t_N for the compensator and the epilogue
  double mu0, tau_x, tau_t, theta, omega, h;
  double t_last;
  double tscale;  // scaled-to-raw time factor of the moments: 1/beta (mixed) or 1 (fp64)
  // per-request float64 constants of the epilogue and compensator (no divisions per row)
  double k_ab;    // A / mu0 = 1 / ((2 pi)^{3/2} tau_x^2 tau_t)
  double k_cw;    // C / theta = omega / (2 pi h^2)
  double inv_tx, inv_tt, inv_h, inv_om;
  // workspace (device)
  double *partials;    // nrt * slices * S * kRowTile
  double *comp;        // nrt * 8: per row tile, the sums of Lambda_n and d Lambda_n / d Theta
                       // (written by slice 0 of the pair kernel), or nullptr (not formed)
  unsigned *rt_count;  // nrt + 1 counters, zero at launch (fused epilogue): finished slices per
                       // row tile, then finished row tiles
  double *rt_sum;      // nrt * 8: per row tile, sum of log lambda_n and of the gradient terms
  double *out;         // 7 doubles: ell, d ell / d Theta
  double *mu_out;      // optional per-event mu_n (n doubles) or nullptr
  double *xi_out;      // optional per-event xi_n (n doubles) or nullptr
};

struct Batch {
  int nreq;
  int total_items;  // pair-kernel items over all requests
  int mode;         // 0 fp64, 1 mixed (one mode per launch)
  int fused;        // 1: the pair kernel finishes each row tile and each request itself
  unsigned *counter;  // pair-kernel work counter, zeroed before the launch
  Request req[kMaxBatch];
};

// Launchers (defined in the kernel translation units). grid is the persistent
// grid size; the kernels loop over items with an atomic counter.
cudaError_t launch_pair_mixed(const Batch &b, bool grad, int grid, cudaStream_t s);
cudaError_t launch_pair_fp64(const Batch &b, bool grad, int grid, cudaStream_t s);
// Resident CTAs per SM of each pair kernel (for the persistent grid and the slices).
int occupancy_pair_mixed(bool grad);
int occupancy_pair_fp64(bool grad);

// Item lookup: the request whose [item_begin, next item_begin) holds `item`.
__host__ __device__ inline int find_request(const Batch &b, int item) {
  int lo = 0, hi = b.nreq - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b.req[mid].item_begin <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

#ifdef __CUDACC__
// First index k in [0, n) with t[k] >= v (strict = false) or t[k] > v (strict = true),
// n if none, for sorted t; computed by one whole warp with 32-way probing (at most
// ceil(log32 n) + 1 rounds of one load per lane). Every lane returns the result.
template <typename TT>
__device__ inline int warp_search(const TT *t, int n, double v, bool strict) {
  const int lane = threadIdx.x & 31;
  int a = 0, b = n;  // the answer lies in [a, b]
  while (a < b) {
    const int step = (b - a + 31) / 32;
    const int p = a + lane * step;
    bool hit = true;
    if (p < b) {
      const double tp = (double)t[p];
      hit = strict ? (tp > v) : (tp >= v);
    }
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (m == 0u) {  // every probe falls before the answer
      a = a + 31 * step + 1;
      continue;
    }
    const int f = __ffs(m) - 1;
    if (f == 0) {
      b = a;
      break;
    }
    const int pf = a + f * step;
    a = a + (f - 1) * step + 1;
    b = min(pf, b);
  }
  return b;
}

// Column-tile window [x, y) of row tile rt for request R: every column outside it is
// more than cut_early before the tile's first row or more than cut_late after its last
// row, so each of its pair terms with the tile's rows is exactly zero. Called by one
// full warp; every lane returns the window.
template <typename TT>
__device__ inline int2 column_window(const Request &R, const TT *t, int rt) {
  const SetView &S = R.set;
  if (R.flags & kFlagDense) return make_int2(0, S.nct);
  const int r0 = rt * kRowTile, r1 = min(r0 + kRowTile, S.n) - 1;
  const int j0 = warp_search(t, S.n, (double)t[r0] - R.cut_early, false);
  const int j1 = warp_search(t, S.n, (double)t[r1] + R.cut_late, true);
  const int c0 = j0 / kColTile;
  const int c1 = min((j1 + kColTile - 1) / kColTile, S.nct);
  return make_int2(c0, max(c1, c0 + 1));
}

__device__ __forceinline__ double std_normal_pdf(double u) {
  return exp(-0.5 * u * u) * 0.39894228040143267794;  // 1 / sqrt(2 pi)
}

// Compensator of Section 2.1 for the rows of row tile rt, summed in a fixed order over the
// CTA: Lambda_n = mu0 (Phi((t_N - t_n)/tau_t) - Phi(-t_n/tau_t)) + theta (1 - e^{-omega (t_N -
// t_n)}) and, with `grad`, its derivatives with respect to (mu0, tau_x, tau_t, theta, omega,
// h). Thread 0 writes the 7 sums to R.comp[8 rt ...]. Called by every thread of the CTA.
template <typename TT>
__device__ void compensator_tile(const Request &R, const TT *t, int rt, bool grad) {
  __shared__ double red[kMaxCtaWarps][8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (blockDim.x + 31) >> 5;
  const double mu0 = R.mu0, th = R.theta, om = R.omega, tN = R.t_last, inv_tt = R.inv_tt;
  double v[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const int end = min((rt + 1) * kRowTile, R.set.n);
  for (int i = rt * kRowTile + tid; i < end; i += blockDim.x) {
    const double tn = (double)t[i];
    const double a = (tN - tn) * inv_tt, b = -tn * inv_tt, D = tN - tn;
    const double e = exp(-om * D);
    const double Pa = normcdf(a), Pb = normcdf(b);
    v[0] += mu0 * (Pa - Pb) + th * (1.0 - e);
    if (grad) {
      v[1] += Pa - Pb;
      v[3] += mu0 * inv_tt * (-a * std_normal_pdf(a) + b * std_normal_pdf(b));
      v[4] += 1.0 - e;
      v[5] += th * D * e;
    }
  }
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    double x = v[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if (lane == 0) red[warp][q] = x;
  }
  __syncthreads();
  if (tid < 7) {
    double x = 0.0;
    for (int w = 0; w < nw; ++w) x += red[w][tid];
    R.comp[(size_t)rt * 8 + tid] = x;
  }
  __syncthreads();
}

// Fused epilogue of row tile rt, run by the CTA that finished its last slice (Section 2.1):
// the row sums over the tile's slices in slice order, lambda_n = A S_b + C S_s, log lambda_n
// and the gradient terms (d lambda_n / d Theta) / lambda_n, summed over the tile's rows in a
// fixed order into R.rt_sum. The CTA that finishes the request's last row tile then writes
// ell = sum over row tiles of (rt_sum - comp), in a fixed order, to R.out. Called by every
// thread of the CTA; the caller has made the slices' partial sums visible (threadfence).
template <bool GRAD>
__device__ void rowtile_epilogue(const Request &R, int rt) {
  constexpr int NS = GRAD ? kSumsGrad : kSumsLoglik;
  constexpr int NV = GRAD ? 7 : 1;
  __shared__ double red2[kMaxCtaWarps][8];
  __shared__ int s_final;
  const SetView &S = R.set;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (blockDim.x + 31) >> 5;
  const double mu0 = R.mu0, th = R.theta;
  const double itx = R.inv_tx, itt = R.inv_tt, ih = R.inv_h, iom = R.inv_om;
  const double Ab = R.k_ab, Cw = R.k_cw, A = mu0 * Ab, C = th * Cw;
  double v[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = 0.0;
  const int r0 = rt * kRowTile, end = min(r0 + kRowTile, S.n);
  for (int i = r0 + tid; i < end; i += blockDim.x) {
    const int li = i - r0;
    double sums[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) sums[s] = 0.0;
    for (int k = rt * R.slices; k < (rt + 1) * R.slices; ++k) {
      const double *src = R.partials + (size_t)k * NS * kRowTile + li;
#pragma unroll
      for (int s = 0; s < NS; ++s) sums[s] += __ldcg(src + s * kRowTile);
    }
    const double mu = A * sums[0], xi = C * sums[1], lam = mu + xi;
    if (R.mu_out) R.mu_out[i] = mu;
    if (R.xi_out) R.xi_out[i] = xi;
    v[0] += log(lam);
    if (GRAD) {
      const double Sb = sums[0], Ss = sums[1], Rb = sums[2], Tb = sums[3] * R.tscale * R.tscale;
      const double Rs = sums[4], Us = sums[5] * R.tscale;
      const double inv = 1.0 / lam;
      v[1] += Ab * Sb * inv;
      v[2] += A * itx * (-2.0 * Sb + Rb * itx * itx) * inv;
      v[3] += A * itt * (-Sb + Tb * itt * itt) * inv;
      v[4] += Cw * Ss * inv;
      v[5] += C * (Ss * iom - Us) * inv;
      v[6] += C * ih * (-2.0 * Ss + Rs * ih * ih) * inv;
    }
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double x = v[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if (lane == 0) red2[warp][q] = x;
  }
  __syncthreads();
  if (tid < NV) {
    double x = 0.0;
    for (int w = 0; w < nw; ++w) x += red2[w][tid];
    R.rt_sum[(size_t)rt * 8 + tid] = x;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_final = atomicAdd(R.rt_count + S.nrt, 1u) == (unsigned)(S.nrt - 1);
  __syncthreads();
  if (s_final) {
    __threadfence();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double x = 0.0;
      for (int r = tid; r < S.nrt; r += blockDim.x)
        x += __ldcg(R.rt_sum + (size_t)r * 8 + q) - __ldcg(R.comp + (size_t)r * 8 + q);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      if (lane == 0) red2[warp][q] = x;
    }
    __syncthreads();
    if (tid < NV) {
      double x = 0.0;
      for (int w = 0; w < nw; ++w) x += red2[w][tid];
      R.out[tid] = x;
    }
  }
  __syncthreads();
}

// End of a pair-kernel item: count the finished slice of row tile rt; the CTA that finishes
// the tile's last slice runs its fused epilogue. Called by every thread of the CTA.
template <bool GRAD>
__device__ void finish_item(const Batch &B, const Request &R, int rt) {
  if (!B.fused) return;
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(R.rt_count + rt, 1u) == (unsigned)(R.slices - 1);
  __syncthreads();
  if (s_last) {
    __threadfence();
    rowtile_epilogue<GRAD>(R, rt);
  }
}
#endif

}  // namespace hk
