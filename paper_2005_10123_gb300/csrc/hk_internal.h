// Internal declarations shared by the kernels and the host runtime of the library.
// Not part of the public ABI (include/hawkes.h is).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hk {

// ---- tiling -------------------------------------------------------------------------
// A pair-kernel CTA holds kRowTile consecutive rows (events n) in registers,
// kRowsPerThread per thread, and streams column tiles of kColTile events (n')
// through shared memory. Event arrays are padded to a multiple of kRowTile.
constexpr int kThreads = 128;
constexpr int kRowsPerThread = 4;
constexpr int kRowTile = kThreads * kRowsPerThread;  // 512
constexpr int kColTile = 256;
constexpr int kWarpRows = 32 * kRowsPerThread;       // 128 consecutive rows per warp
constexpr int kEpiThreads = 256;                     // epilogue rows per CTA
constexpr int kMaxBatch = 64;                        // requests per launch
constexpr int kSumsLoglik = 2;                       // S_b, S_s
constexpr int kSumsGrad = 6;                         // S_b, S_s, R_b, T_b, R_s, U_s

// Sentinel for padded events: a time so large that every pair term involving a
// padded event is exactly zero (its squared time distance overflows to +inf).
constexpr float kPadTime32 = 1.0e30f;
constexpr double kPadTime64 = 1.0e300;

// One resident event set, as the kernels see it.
struct SetView {
  const float *x32, *y32, *t32;
  const double *x64, *y64, *t64;
  const int *lo32, *lo64;  // lo[i] = first index with the same stored time as event i
  int n, npad, nrt, nct;   // events, padded length, row tiles, column tiles
};

// Work schedule of one request kind on one set. A "piece" is a run of column tiles
// of one row tile; pieces are sorted by (row tile, first column tile), so the piece
// index is also the partial-sum slot and slot_first[rt] is the first piece of row
// tile rt. A "range" (one work item of the persistent pair kernel) is a run of
// consecutive pieces of about equal cost.
struct Schedule {
  const int4 *pieces;      // {row_tile, col_tile_begin, col_tile_end, 0}
  const int *range_first;  // nranges + 1
  const int *slot_first;   // nrt + 1
  int npieces, nranges;
};

struct Request {
  SetView set;
  Schedule sched;
  int grad;        // 0: loglik only; 1: loglik and gradient
  int flags;       // HAWKES_FLAG_* of the context at submission
  int item_begin;  // first pair-kernel item (range) of this request in the batch
  int epi_begin;   // first epilogue item (block of kEpiThreads rows) in the batch
  // float32 pair constants (mixed mode)
  float a2;    // log2(e) / (2 tau_x^2)                  multiplies raw r^2
  float beta;  // sqrt(log2(e) / (2 tau_t^2))            scales (t - t0)
  float wn;    // -omega log2(e) / beta                  multiplies scaled dt
  float cn;    // -log2(e) / (2 h^2)                     multiplies raw r^2
  // float64 pair constants (fp64 mode)
  double da;   // 1 / (2 tau_x^2)
  double db;   // 1 / (2 tau_t^2)
  double dc;   // 1 / (2 h^2)
  // Theta and t_N for the epilogue
  double mu0, tau_x, tau_t, theta, omega, h;
  double t_last;
  double tscale;  // scaled-to-raw time factor of the moments: 1/beta (mixed) or 1 (fp64)
  // workspace (device)
  double *partials;    // npieces * S * kRowTile
  double *block_part;  // epilogue blocks * 8
  unsigned *ticket;    // epilogue completion counter, zero between launches
  double *out;         // 7 doubles: ell, d ell / d Theta
  double *mu_out;      // optional per-event mu_n (n doubles) or nullptr
  double *xi_out;      // optional per-event xi_n (n doubles) or nullptr
};

struct Batch {
  int nreq;
  int total_items;  // pair-kernel items (ranges) over all requests
  int total_epi;    // epilogue items over all requests
  int mode;         // 0 fp64, 1 mixed (one mode per launch)
  unsigned *counter;  // pair-kernel work counter, zeroed before the launch
  Request req[kMaxBatch];
};

// Launchers (defined in the kernel translation units). grid is the persistent
// grid size; the kernels loop over items with an atomic counter.
cudaError_t launch_pair_mixed(const Batch &b, bool grad, int grid, cudaStream_t s);
cudaError_t launch_pair_fp64(const Batch &b, bool grad, int grid, cudaStream_t s);
cudaError_t launch_epilogue(const Batch &b, bool grad, int grid, cudaStream_t s);
// Resident CTAs per SM of each pair kernel (for the persistent grid and schedule).
int occupancy_pair_mixed(bool grad);
int occupancy_pair_fp64(bool grad);

// Item lookup: the request whose [begin, next begin) holds `item`.
__host__ __device__ inline int find_request(const Batch &b, int item, bool epi) {
  int lo = 0, hi = b.nreq - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    int start = epi ? b.req[mid].epi_begin : b.req[mid].item_begin;
    if (start <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace hk
