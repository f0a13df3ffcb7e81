// Internal declarations shared by the kernels and the host runtime of the library.
// Not part of the public ABI (include/hawkes.h is).
#pragma once

#include <cmath>
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
#define HK_THREADS 64  // two warps: the per-tile barrier waits on one other warp only
#endif
#ifndef HK_COL_TILE
#define HK_COL_TILE 128
#endif
constexpr int kThreads = HK_THREADS;
constexpr int kRowsPerThread = HK_ROWS_PER_THREAD;  // even: rows are processed in packed pairs
constexpr int kRowTile = kThreads * kRowsPerThread;  // 256: 64 threads x 4 rows
constexpr int kColTile = HK_COL_TILE;
constexpr int kWarpRows = 32 * kRowsPerThread;       // consecutive rows per warp
constexpr int kPadTo = kRowTile > kColTile ? kRowTile : kColTile;  // event arrays padded to this
#ifndef HK_SYM_NEAR
#define HK_SYM_NEAR 1  // shared background: share the near column tiles before a row tile too
#endif
#ifndef HK_SYM_DESC
#define HK_SYM_DESC 1  // shared-background launches: row tiles latest first (see item_at)
#endif
constexpr int kEpiThreads = 256;                     // rows per CTA of the allocation-free epilogue
constexpr int kMaxBatch = 64;                        // requests per launch
constexpr int kSumsLoglik = 2;                       // S_b, S_s
constexpr int kSumsGrad = 6;                         // S_b, S_s, R_b, T_b, R_s, U_s
// Mixture of triggering functions (the extension of the paper's Discussion): MIX components, each
// with its own (theta, omega, h); component 2 adds a trigger sum (and two moments) per row.
constexpr int kMixMax = 2;
// Row sums of a kernel: S_b, S_s1[, S_s2] (loglik); S_b, S_s1, R_b, T_b, R_s1, U_s1[, S_s2, R_s2, U_s2]
__host__ __device__ constexpr int num_sums(bool grad, int mix) { return grad ? 3 + 3 * mix : 1 + mix; }
constexpr int kMaxSums = num_sums(true, kMixMax);
// Gradient entries: (mu0, tau_x, tau_t) and (theta, omega, h) per component.
__host__ __device__ constexpr int num_grad(int mix) { return 3 + 3 * mix; }
constexpr int kOut = 16;  // doubles per request in out, comp and rt_sum: ell, then up to 9 gradient terms
constexpr int kFlagExcludeSelf = 1;                  // HAWKES_FLAG_EXCLUDE_SELF
constexpr int kFlagDense = 2;                        // HAWKES_FLAG_DENSE
constexpr int kFlagNoSymmetry = 4;                   // HAWKES_FLAG_NO_SYMMETRY
constexpr int kFlagTestWithholdReady = 1 << 30;      // HAWKES_FLAG_TEST_WITHHOLD_READY (tests only)
constexpr unsigned kStatusMergeTimeout = 1u;         // Request::status: a merge-tree wait ran out
constexpr unsigned kStatusFixRange = 2u;             // Request::status: a sum left the fixed-point range
                                                     // (not finite, or |v 2^F| >= 2^62): results NaN
// widest pair-kernel CTA: the grouped kernel's, two rows per thread
constexpr int kMaxCtaWarps = (kRowTile / 2 > kThreads ? kRowTile / 2 : kThreads) / 32;
static_assert(kThreads <= 32 * kMaxCtaWarps && kRowTile / 4 <= 32 * kMaxCtaWarps, "CTA too wide");

// Column-tile lookup by time, built once per event set and precision: time is cut into nb
// equal buckets, bucket b = [t0 + b / inv, t0 + (b + 1) / inv). first[b] counts the column
// tiles whose latest time lies below the start of bucket b, last[b] the column tiles whose
// earliest time is at most the end of bucket b. A column window [tau0, tau1] in time then maps
// to a superset of its column tiles with two table reads (see table_window).
struct WinTable {
  const int *first, *last;
  double t0, inv;
  int nb;  // 0: no table
};
constexpr int kWinBuckets = 4096;

// One resident event set, as the kernels see it.
struct SetView {
  const float *x32, *y32, *t32;
  const double *x64, *y64, *t64;
  const int *lo32, *lo64;  // lo[i] = first index with the same stored time as event i
  WinTable win32, win64;   // column-tile lookups over the float32 and float64 times
  int n, npad, nrt, nct;   // events, padded length, row tiles, column tiles
};

// Column tiles [x, y) that hold every column with time in [tau0, tau1] (a superset by at most
// the columns of two buckets on each side; columns outside the exact range only add exact
// zeros). One bucket of margin on each side absorbs the rounding of the bucket index.
// The first column tile of such a window: every column tile before it holds only times below
// tau0.
__host__ __device__ inline int table_first(const WinTable &W, double tau0) {
  const double u0 = (tau0 - W.t0) * W.inv;
  if (!(u0 >= 1.0)) return 0;
  const double b = floor(u0) - 1.0;
  return W.first[b >= (double)(W.nb - 1) ? W.nb - 1 : (int)b];
}

__host__ __device__ inline int2 table_window(const WinTable &W, int n, int nct, double tau0, double tau1) {
  const int real = (n + kColTile - 1) / kColTile;  // column tiles holding real events
  int c1 = real;
  const int c0 = table_first(W, tau0);
  const double u1 = (tau1 - W.t0) * W.inv;
  if (u1 < (double)(W.nb - 1)) c1 = W.last[u1 < 0.0 ? 0 : (int)floor(u1) + 1];
  c1 = c1 < nct ? c1 : nct;
  return make_int2(c0, c1 > c0 + 1 ? c1 : c0 + 1);
}

// Work decomposition: the pair kernels run one CTA per item. A request's items are first
// one compensator item per row tile (when comp is set), then the pair items. For a pair item
// the kernel finds the window of column tiles of its row tile rt that can hold a nonzero pair
// term that matters (with the self term, every other pair term is below 2^-40 (mixed) or 2^-70
// (float64) of lambda_n / N; without it, exactly zero; see cut_early and cut_late) and cuts it into `slices`
// near-equal leaves. Row tiles are launched from the
// middle of the time range outwards; one item covers `span` consecutive leaves of its row
// tile, with span 4 for the first `wide` row tiles launched, 2 up to `coarse` and 1 for the
// rest, so that the launch starts on long items and ends on short ones. Items are numbered in
// launch order; the item's number is its partial-sum slot, so results do not depend on which
// CTA ran which item or when. An unfused launch (Batch::fused = 0, 1-leaf items only) leaves
// each item's sums in the row-tile-major slot rt * slices + leaf for a separate epilogue.
struct Request {
  SetView set;
  int slices;      // leaves per row tile (fixed per set and kernel kind)
  int wide;        // row tiles launched first whose items span 4 leaves
  int coarse;      // row tiles launched before the 1-leaf items (span 4 or 2)
  int grad;        // 0: loglik only; 1: loglik and gradient
  int flags;       // HAWKES_FLAG_* of the context at submission
  int item_begin;  // first pair-kernel item of this request in the batch
  // Column window: column n' can only contribute to row n if
  //   t_n - cut_early <= t_n' <= t_n + cut_late   (days; +inf keeps every column)
  double cut_early, cut_late;
  // float32 pair constants (mixed mode). The two scales applied to stored values (s to the
  // coordinates of background-only tiles, beta to times) are each held as a float32 head and
  // tail, v = hi + lo to about 2^-48 relative, so that a scaled value is the correctly rounded
  // product with the float64 scale (scale_split): a float32-rounded bandwidth would shift every
  // pair term the same way, and where a gradient component nearly cancels (d ell / d tau_t on the
  // N = 85,000 workload cancels to about 2e-3 per row) that shift dominates its error.
  float a2;              // log2(e) / (2 tau_x^2), rounded       multiplies r^2 (tiles with trigger terms)
  float s_hi, s_lo;      // s = sqrt(a2)                         scales x, y (background-only tiles)
  float beta, beta_lo;   // beta = sqrt(log2(e) / (2 tau_t^2))   scales (t - t0)
  float b2, b2_lo;       // beta^2 = b2 + b2_lo                  multiplies dt^2 (grouped kernel)
  float wn;              // -omega log2(e) / beta                scaled dt: tile classes (the mixed
                         //                                      kernel's terms use -omega log2(e))
  float cn;              // -log2(e) / (2 h^2)                   multiplies r^2
  int mix;               // trigger components: 1 (Section 2.1) or 2 (mixture; Batch::mix2)
  // float64 pair constants (fp64 mode)
  double da;   // 1 / (2 tau_x^2)
  double db;   // 1 / (2 tau_t^2)
  double dc;   // 1 / (2 h^2)
  // Theta and t_N for the compensator and the epilogue
  double mu0, tau_x, tau_t, theta, omega, h;
  double t_last;
  double tscale;  // scaled-to-raw time factor of the moments: 1/beta (mixed) or 1 (fp64)
  double inv_a2;  // 1 / a2 in float64: R_b = (Q - T_b) / a2 from the background moment Q (mixed)
  // per-request float64 constants of the epilogue and compensator (no divisions per row)
  double k_ab;    // A / mu0 = 1 / ((2 pi)^{3/2} tau_x^2 tau_t)
  double k_cw;    // C / theta = omega / (2 pi h^2)
  double inv_tx, inv_tt, inv_h, inv_om;
  // workspace (device)
  double *partials;    // one slot of S * kRowTile float64 row sums per pair item
  double *comp;        // nrt * kOut: per row tile, the sums of Lambda_n and d Lambda_n / d Theta
                       // (written by the compensator items), or nullptr (not formed)
  unsigned *rt_count;  // request_counters(R) counters, zero at launch (fused epilogue): the
                       // merge-tree nodes of every row tile (2 slices from 2 rt slices), then
                       // the finished row-tile epilogues and compensator items
  double *rt_sum;      // nrt * kOut: per row tile, sum of log lambda_n and of the gradient terms
  // symmetric background (see SymPlan): far column tiles share each background term between its
  // row and its column. Every event's sums, from its row's items and from the far column tiles
  // holding it, go to fixsum as exact fixed-point integers (no partial-sum slots, no merge tree).
  int sym;             // 1: on (mixed, fused, set with a time table, no exclude-self/dense/no-symmetry);
                       // 2: the near column tiles before the row tile shared too
  signed char fix_bits[kMaxSums];  // sym: sum s enters fixsum as round(v 2^fix_bits[s]) (fix_bits_for)
  double trig_cut;     // days: columns earlier than t_n - trig_cut give trigger terms that contribute
                       // nothing (with the self term below 2^-40 (mixed) or 2^-70 (float64) of
                       // lambda_n in all; without it exact zeros)
  long long *fixsum;   // sym, or a grouped batch without exclude-self: [num_sums][npad] per-event sums
                       // in fixed point, zero at launch (nullptr: partial-sum slots and merge trees)
  unsigned *rt_done;   // with fixsum: per row tile, the arrivals of its items (and, with sym, of the
                       // far column tiles holding its columns), zero at launch
  double *out;         // ell, then d ell / d Theta (6 entries, 9 for a two-component mixture)
  unsigned *status;    // device word, zero at launch: kStatusMergeTimeout if a device wait of
                       // this request ran out (its results are then NaN), or nullptr
  double *mu_out;      // optional per-event mu_n (n doubles) or nullptr
  double *xi_out;      // optional per-event xi_n (n doubles) or nullptr
  double *pi_out;      // optional per-event pi_n = xi_n / lambda_n (n doubles) or nullptr
};

// Component 2 of a two-component trigger mixture. A mixture launch holds one request, so its
// second component's constants sit in the Batch (kernel parameters are limited to 32 KB).
struct MixConst {
  float wn2, cn2;          // as Request::wn, cn
  double theta2, omega2, h2;
  double dc2;              // 1 / (2 h_2^2)
  double k_cw2, inv_h2, inv_om2;
};

struct Batch {
  MixConst mix2;  // used when a request has mix = 2
  int nreq;
  int total_items;  // pair-kernel items (= CTAs) over all requests
  int mode;         // 0 fp64, 1 mixed (one mode per launch)
  int fused;        // 1: the pair kernel finishes each row tile and each request itself
  int group;        // 0, or the grouped kernel's group size (every request on one set)
  int comp_total;   // grouped kernel: compensator items, first in the launch
  int split;        // 1: requests with the shared background (sym) leave their epilogues to
                    // epilogue_fix_kernel, launched after the pair kernel (see launch_epilogue_fix)
  Request req[kMaxBatch];
};

// The split epilogue (Batch::split): one CTA of kEpiRows threads per kEpiRows consecutive events
// of each request with the shared background, one event per thread; its partial sums go to
// rt_sum[block] (a request's rt_sum holds 3 nrt slots: its epi_blocks, at most 2 nrt, then the
// sums of groups of 32 blocks from slot 2 nrt on), and the groups' counters are the first of
// the request's merge-tree counters, which the shared background does not use.
constexpr int kEpiRows = 128;
__host__ __device__ inline int epi_blocks(const Request &R) { return (R.set.n + kEpiRows - 1) / kEpiRows; }

// The mixed-precision constants of a request from Theta (Section 2.1, d = 2; base-2 exponents):
// e_b = 2^-(a2 r^2 + beta^2 dt^2), e_s = 2^(cn r^2 + wn beta dt). Host code.
inline void set_mixed_constants(Request *R, double tau_x, double tau_t, double omega, double h) {
  const double log2e = 1.4426950408889634074;
  const double a2 = log2e / (2.0 * tau_x * tau_x), s = std::sqrt(a2);
  const double beta = std::sqrt(log2e / (2.0 * tau_t * tau_t));
  R->a2 = (float)a2;
  R->s_hi = (float)s;
  R->s_lo = (float)(s - (double)R->s_hi);
  R->beta = (float)beta;
  R->beta_lo = (float)(beta - (double)R->beta);
  R->b2 = (float)(beta * beta);
  R->b2_lo = (float)(beta * beta - (double)R->b2);
  R->wn = (float)(-omega * log2e / beta);
  R->cn = (float)(-log2e / (2.0 * h * h));
  R->inv_a2 = 1.0 / a2;
  R->tscale = 1.0 / beta;
}

// Items of one request (see Request): compensator items first, then pair items.
__host__ __device__ inline int comp_items(const Request &R) { return R.comp ? R.set.nrt : 0; }
// Leaves per item of the row tile launched k-th (see Request).
__host__ __device__ inline int span_at(const Request &R, int k) { return k < R.wide ? 4 : k < R.coarse ? 2 : 1; }
__host__ __device__ inline int pair_items(const Request &R) {
  const int K = R.slices;
  return R.wide * ((K + 3) / 4) + (R.coarse - R.wide) * ((K + 1) / 2) + (R.set.nrt - R.coarse) * K;
}
__host__ __device__ inline int request_items(const Request &R) { return comp_items(R) + pair_items(R); }
// Merge-tree nodes (fewer than 2 per leaf) of every row tile, then the final counter.
__host__ __device__ inline int request_counters(const Request &R) { return 2 * R.set.nrt * R.slices + 1; }
// The scales of a grouped-kernel request (pair_group.cu), whose moments are in raw units:
// R_b = sum r^2 e_b with r^2 e^(-r^2 / (2 tau_x^2)) <= 2 tau_x^2 / e, and T_b = sum dt^2 e_b with
// dt^2 e^(-dt^2 / (2 tau_t^2)) <= 2 tau_t^2 / e.
inline void set_fix_bits_raw(Request *R, int grad, double span);
// Pair items of a row tile whose items span `span` leaves each.
__host__ __device__ inline int rowtile_items(const Request &R, int span) { return (R.slices + span - 1) / span; }

// Fixed-point scales of the per-event sums (Request::fixsum). A sum over at most npad terms, each
// at most B, stays below 2^62 as round(v 2^F) when 2^F <= 2^62 / (npad B); F = 62 - ceil(log2
// npad) - ceil(log2 B). The per-term bounds B, in the units the kernels accumulate:
//   S_b, S_s: 1 (terms 2^-q, q >= 0);  Q = sum q 2^-q and T_b = sum u 2^-q with 0 <= u <= q:
//   q 2^-q <= 1 / (e ln 2) < 1;  R_s = sum r^2 e_s: r^2 2^(cn r^2) <= 2 h^2 / e;
//   U_s = sum dt e_s (units of time): dt e^(-omega dt) <= min(1 / (e omega), span of the times).
// The absolute resolution 2^-F is about npad B 2^-62 (2.8e-14 for S_b at N = 85,000, against a
// floor of 1 for the self term, so S_b keeps 14 digits; every other sum enters lambda_n and the
// gradient through ratios to lambda_n, so its absolute resolution is what matters).
inline int fix_bits_for(int64_t npad, double bound) {
  int bits = 0;
  while (((int64_t)1 << bits) < npad) ++bits;
  int b = 0;
  if (bound > 1.0) b = (int)std::ceil(std::log2(bound));
  else if (bound > 0.0) b = -(int)std::floor(-std::log2(bound));  // ceil(log2 bound) <= 0
  const int F = 62 - bits - b;
  return F < -100 ? -100 : F > 120 ? 120 : F;
}
// The fixed-point scales of one request: component c's trigger sums with its own h and omega.
inline void set_fix_bits(Request *R, int grad, int mix, double h1, double om1, double h2, double om2, double span) {
  const double e = 2.71828182845904523536;
  const int64_t np = R->set.npad;
  for (int s = 0; s < kMaxSums; ++s) R->fix_bits[s] = (signed char)fix_bits_for(np, 1.0);
  if (!grad) return;
  auto rs = [&](double h) { return 2.0 * h * h / e; };
  auto us = [&](double om) { return std::fmin(1.0 / (e * om), span > 0.0 ? span : 1.0); };
  R->fix_bits[4] = (signed char)fix_bits_for(np, rs(h1));
  R->fix_bits[5] = (signed char)fix_bits_for(np, us(om1));
  if (mix > 1) {
    R->fix_bits[7] = (signed char)fix_bits_for(np, rs(h2));
    R->fix_bits[8] = (signed char)fix_bits_for(np, us(om2));
  }
}
inline void set_fix_bits_raw(Request *R, int grad, double span) {
  set_fix_bits(R, grad, 1, R->h, R->omega, 0.0, 0.0, span);
  if (!grad) return;
  const double e = 2.71828182845904523536;
  R->fix_bits[2] = (signed char)fix_bits_for(R->set.npad, 2.0 * R->tau_x * R->tau_x / e);
  R->fix_bits[3] = (signed char)fix_bits_for(R->set.npad, 2.0 * R->tau_t * R->tau_t / e);
}

// The request's p-th pair item in launch order: row tile rt, index `node` among the row tile's
// items, leaves [node * span, min(node * span + span, slices)), and `base`, the slot of the row
// tile's first item (the item's own slot is base + node = p). Row tiles go out from the middle
// of the time range (m, m - 1, m + 1, m - 2, ...): the first and last row tiles, whose column
// windows are cut off by t = 0 and t = t_N, launch last. With the shared background (R.sym) they
// go out latest first: a row tile's far contributors are the later row tiles, which then launch
// before it, and the launch ends on the earliest row tiles, whose windows t = 0 cuts short.
struct PairItem {
  int rt, node, span, base;
};
// Launch position k of row tile rt (the inverse of the middle-out order of item_at) and the
// number of its first pair item (its `base`).
__host__ __device__ inline int first_item_of(const Request &R, int rt) {
  const int m = R.set.nrt / 2;
  const int k = R.sym && HK_SYM_DESC ? R.set.nrt - 1 - rt : rt == m ? 0 : rt < m ? 2 * (m - rt) - 1 : 2 * (rt - m);
  const int K = R.slices, n4 = (K + 3) / 4, n2 = (K + 1) / 2;
  if (k < R.wide) return k * n4;
  if (k < R.coarse) return R.wide * n4 + (k - R.wide) * n2;
  return R.wide * n4 + (R.coarse - R.wide) * n2 + (k - R.coarse) * K;
}

// ---- symmetric background ----------------------------------------------------------------
// A background term e_b(n, n') = e_b(n', n) serves the rows of both events. With R.sym, a row
// tile K evaluates the column tiles J of its window that lie beyond the trigger's reach (no
// trigger term of K's rows with them can change the sums, see trig_cut) once, adding each term
// to its row
// and to its column. Those "far" column tiles are [c0(K), 2 ib(K)):
//   c0(K) = table_first(t_K - cut_early), ib(K) = table_first(t_K - trig_cut) / 2,
// with t_K the time of row tile K's first event; they end on a row-tile boundary, so a far
// block always covers whole row tiles' columns. Every other pair is evaluated row by row as
// before: row tile I visits the column tiles [max(c0(I), 2 ib(I)), min(c1(I), 2 kmax(I) + 2)),
// kmax(I) = the last row tile K with ib(K) <= I (the later row tiles for which I is not far).
// A pair (n in I, n' in K > I) is so covered exactly once in each direction: by K's far block
// when I < ib(K), else by I's late columns (K <= kmax(I)) and K's near early columns. With
// R.sym == 2 (sym_plan_near) K's near early columns [sym_end(K), 2 K) serve both directions too,
// and I's late columns are not visited.
// Every event's sums reach R.fixsum as integers round(v 2^F) (fix_bits_for): each item adds its
// rows' float64 sums, each far block its columns' float32 sums. Integer additions commute
// exactly, so the totals do not depend on the order in which items finish. The pair kernel's
// items only add; the batch's split epilogue (epilogue_fix_kernel, Batch::split), launched after
// it on the same stream, turns the totals into every event's terms, so no item waits for or
// counts another. e_col(I), the far column tiles of later row tiles that hold I's columns, is
// part of the plan the host tests check block by block.
// kSymRootMark: the grouped kernel's row-tile counters (pair_group.cu) count to it.
constexpr unsigned kSymRootMark = 1u << 30;

struct SymK {
  int c0, ib;  // first window column tile and first non-far row tile of row tile K
};
__host__ __device__ inline SymK sym_k(const Request &R, const WinTable &W, double t_first) {
  return SymK{table_first(W, t_first - R.cut_early), table_first(W, t_first - R.trig_cut) / 2};
}

// The plan of row tile I: far column tiles [c0, sym_end), shared near ones [sym_end, near_end)
// (R.sym == 2; empty otherwise), near ones evaluated row by row [near_end, end), and e_col, the
// far column tiles of later row tiles that hold I's columns.
struct SymPlan {
  int sym_end, near_end, end, e_col;
};

// One row tile K's contribution to the plan of row tile I < K: its far column tiles among I's
// two column tiles (e_col), and whether I is near for K (then I's near columns reach into K).
__host__ __device__ inline void sym_visit(const SymK &k, int I, int *e_col, bool *near) {
  *e_col += (k.c0 <= 2 * I && 2 * I < 2 * k.ib) + (k.c0 <= 2 * I + 1 && 2 * I + 1 < 2 * k.ib);
  *near = k.ib <= I;
}
// Later row tiles K stop mattering to I once both hold: K's window starts after I's columns and
// I is far for K (c0 and ib are non-decreasing in K).
__host__ __device__ inline bool sym_done(const SymK &k, int I) { return k.c0 > 2 * I + 1 && k.ib > I; }

// With R.sym == 2 the near column tiles before row tile I's own, [sym_end, 2 I), are shared as
// well: their background terms serve both events, their trigger terms the rows. Row tile I then
// visits its own two column tiles and no later ones row by row, because every later row tile K
// for which I is near (ib(K) <= I) holds I's columns among its shared near tiles.
__host__ __device__ inline SymPlan sym_plan_near(int2 win, int sym_end, int I, int e_col) {
  const int own = 2 * I < win.y ? 2 * I : win.y;
  const int near_end = own > sym_end ? own : sym_end;
  const int end = win.y < 2 * I + 2 ? win.y : 2 * I + 2;
  return SymPlan{sym_end, near_end, end, e_col};
}

// The plan of row tile I from its window [c0, c1) (table_window_rt), by a plain scan over the
// later row tiles; tfirst(K) is row tile K's first event time. Host code and reference for the
// kernels' warp-parallel version.
template <class TFirst>
__host__ __device__ inline SymPlan sym_plan_scan(const Request &R, const WinTable &W, int I, int2 win, TFirst tfirst) {
  const SymK own = sym_k(R, W, tfirst(I));
  int e_col = 0, kmax = I;
  for (int K = I + 1; K < R.set.nrt; ++K) {
    const SymK k = sym_k(R, W, tfirst(K));
    if (sym_done(k, I)) break;
    bool near;
    sym_visit(k, I, &e_col, &near);
    if (near) kmax = K;
  }
  const int sym_end = win.x > 2 * own.ib ? win.x : 2 * own.ib;
  if (R.sym == 2) return sym_plan_near(win, sym_end, I, e_col);
  const int end = win.y < 2 * kmax + 2 ? win.y : 2 * kmax + 2;
  return SymPlan{sym_end, sym_end, end, e_col};
}
__host__ __device__ inline PairItem item_at(const Request &R, int p) {
  const int K = R.slices, n4 = (K + 3) / 4, n2 = (K + 1) / 2;
  const int p2 = R.wide * n4, p1 = p2 + (R.coarse - R.wide) * n2;  // first 2-leaf and 1-leaf items
  int k, node, span;
  if (p < p2) { k = p / n4; node = p - k * n4; span = 4; }
  else if (p < p1) { k = (p - p2) / n2; node = p - p2 - k * n2; k += R.wide; span = 2; }
  else { k = (p - p1) / K; node = p - p1 - k * K; k += R.coarse; span = 1; }
  const int m = R.set.nrt / 2;
  const int rt = R.sym && HK_SYM_DESC ? R.set.nrt - 1 - k : k == 0 ? m : (k & 1) ? m - (k + 1) / 2 : m + k / 2;
  return PairItem{rt, node, span, p - node};
}

// Launchers (defined in the kernel translation units): one CTA per item, grid =
// b.total_items.
cudaError_t launch_pair_mixed(const Batch &b, bool grad, cudaStream_t s);
// With b.split: the epilogues of the batch's sym requests (epilogue_fix_kernel), after the pair
// kernel on the same stream; nothing to launch when no request has sym.
cudaError_t launch_epilogue_fix(const Batch &b, bool grad, cudaStream_t s);
// The split epilogue's log table on the current device (once per context, before any launch).
cudaError_t init_log_table();
cudaError_t launch_pair_fp64(const Batch &b, bool grad, cudaStream_t s);
// Grouped mixed kernel (pair_group.cu): requests on one set in groups of G = b.group, each
// pair's geometry shared by the group. Items: nreq * nrt compensator items, then
// ceil(nreq / G) * nrt * slices pair items. G must be one of kGroupSizes(grad).
cudaError_t launch_pair_group(const Batch &b, bool grad, cudaStream_t s);
// The group sizes the grouped kernel is built for; the largest of each was tuned on 64 requests
// at N = 85,000 (4 with the gradient at 4 resident CTAs per SM, 8 for the log-likelihood).
constexpr int kGroupSizesGrad[] = {4};
constexpr int kGroupSizesLoglik[] = {4, 8};
// Group size for a batch of k requests: a group forms each pair's geometry once (about 6 float32
// operations) and then about 6 (gradient) or 5 (log-likelihood) per request and term, and a
// partial last group evaluates its missing members as copies of its first. The size minimises
// ceil(k / G) (6 + c G) over the built sizes, larger G on ties (64 requests: 4 and 8; 17
// log-likelihood requests: 4, where groups of 8 would evaluate 7 copies).
inline int group_size(bool grad, int k) {
  const int c = grad ? 6 : 5;
  const int *sizes = grad ? kGroupSizesGrad : kGroupSizesLoglik;
  const int count = grad ? (int)(sizeof(kGroupSizesGrad) / sizeof(int)) : (int)(sizeof(kGroupSizesLoglik) / sizeof(int));
  int best = sizes[0];
  long long best_cost = -1;
  for (int i = 0; i < count; ++i) {
    const int G = sizes[i];
    const long long cost = (long long)((k + G - 1) / G) * (6 + c * G);
    if (best_cost < 0 || cost <= best_cost) {
      best = G;
      best_cost = cost;
    }
  }
  return best;
}
// Resident CTAs per SM of each pair kernel (sets the number of slices).
int occupancy_pair_mixed(bool grad);
int occupancy_pair_fp64(bool grad);
// Column chunks per column tile in the float64 kernel's slices (a slice may be shorter than a
// column tile there).
int fp64_chunks_per_tile();

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
  const int c0 = min(j0 / kColTile, S.nct - 1);  // in range even for times a caller left unsorted
  const int c1 = min((j1 + kColTile - 1) / kColTile, S.nct);
  return make_int2(c0, max(c1, c0 + 1));
}

// Column window of row tile rt from the set's lookup table W over times t: every thread of
// the CTA gets the same window without a search or a barrier. (-1, -1) when the set has no
// table (the caller then runs column_window).
template <typename TT>
__device__ inline int2 table_window_rt(const Request &R, const WinTable &W, const TT *t, int rt) {
  const SetView &S = R.set;
  if (R.flags & kFlagDense) return make_int2(0, S.nct);
  if (W.nb == 0) return make_int2(-1, -1);
  const int r0 = rt * kRowTile, r1 = min(r0 + kRowTile, S.n) - 1;
  return table_window(W, S.n, S.nct, (double)__ldg(t + r0) - R.cut_early, (double)__ldg(t + r1) + R.cut_late);
}

__device__ __forceinline__ double std_normal_pdf(double u) {
  return exp(-0.5 * u * u) * 0.39894228040143267794;  // 1 / sqrt(2 pi)
}

// Compensator of Section 2.1 for the rows of row tile rt, summed in a fixed order over the
// CTA: Lambda_n = mu0 (Phi((t_N - t_n)/tau_t) - Phi(-t_n/tau_t)) + theta (1 - e^{-omega (t_N -
// t_n)}) (plus theta_2 (1 - e^{-omega_2 (t_N - t_n)}) for a mixture) and, with `grad`, its
// derivatives in the gradient order (mu0, tau_x, tau_t, theta, omega, h[, theta_2, omega_2,
// h_2]). Thread 0 writes the sums to R.comp[kOut rt ...]. Called by every thread of the CTA of
// a compensator item; these items come first in a request, so their float64 work overlaps the
// pair items instead of ending the launch.
// Scratch of the CTA-wide float64 reductions (compensator_tile, rowtile_reduce, finish_request):
// one array per kernel, reused in turn (each use starts after a barrier and ends with one), so
// that the three cost the pair kernels' occupancy one small array. Row w of the warps' partial
// sums starts at w * kRedWidth; the totals follow the kMaxCtaWarps rows.
constexpr int kRedWidth = 1 + num_grad(kMixMax);  // most values reduced at once
__device__ __forceinline__ double *reduce_scratch() {
  __shared__ double buf[(kMaxCtaWarps + 1) * kRedWidth];
  return buf;
}

template <int MIX = 1, typename TT>
__device__ void compensator_tile(const Request &R, const MixConst &M2, const TT *t, int rt, bool grad) {
  constexpr int NC = 1 + num_grad(MIX);
  static_assert(NC <= kRedWidth, "reduction scratch too narrow");
  double *red = reduce_scratch();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (blockDim.x + 31) >> 5;
  const double mu0 = R.mu0, th = R.theta, om = R.omega, tN = R.t_last, inv_tt = R.inv_tt;
  const double th2 = M2.theta2, om2 = M2.omega2;
  const int nv = grad ? NC : 1;
  double v[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) v[q] = 0.0;
  const int end = min((rt + 1) * kRowTile, R.set.n);
  for (int i = rt * kRowTile + tid; i < end; i += blockDim.x) {
    const double tn = (double)t[i];
    const double a = (tN - tn) * inv_tt, b = -tn * inv_tt, D = tN - tn;  // a >= 0 >= b
    // Far from both ends of [0, t_N] the terms are constants in float64, so most events skip
    // the special functions: e^{-omega D} underflows to 0 beyond omega D = 746; Phi(a) rounds
    // to 1 for a >= 9 (1 - Phi(9) = 1.1e-19), and Phi(b) <= 1.1e-19 vanishes against
    // Phi(a) >= 1/2; the dropped a phi(a) terms are below 1e-17 each.
    const double e = om * D > 746.0 ? 0.0 : exp(-om * D);
    const double Pa = a >= 9.0 ? 1.0 : normcdf(a), Pb = b <= -9.0 ? 0.0 : normcdf(b);
    v[0] += mu0 * (Pa - Pb) + th * (1.0 - e);
    if (grad) {
      const double qa = a >= 9.0 ? 0.0 : a * std_normal_pdf(a), qb = b <= -9.0 ? 0.0 : b * std_normal_pdf(b);
      v[1] += Pa - Pb;
      v[3] += mu0 * inv_tt * (-qa + qb);
      v[4] += 1.0 - e;
      v[5] += th * D * e;
    }
    if constexpr (MIX > 1) {  // component 2 of a mixture
      const double e2 = om2 * D > 746.0 ? 0.0 : exp(-om2 * D);
      v[0] += th2 * (1.0 - e2);
      if (grad) {
        v[7] += 1.0 - e2;
        v[8] += th2 * D * e2;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    double x = v[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if (lane == 0) red[warp * kRedWidth + q] = x;
  }
  __syncthreads();
  if (tid < nv) {
    double x = 0.0;
    for (int w = 0; w < nw; ++w) x += red[w * kRedWidth + tid];
    R.comp[(size_t)rt * kOut + tid] = x;
  }
  __syncthreads();
}

// Count one finished row-tile epilogue or compensator item of request R; the CTA that
// finishes the last of them writes ell = sum over row tiles of (rt_sum - comp) and the
// gradient, in a fixed order, to R.out (NaN if a sum of the request left the fixed-point range,
// kStatusFixRange). Called by every thread of the CTA after its results are written.
// With nsum >= 0 (the split epilogue) the parts are the request's nsum epilogue blocks, whose
// sums sit in rt_sum[0, nsum), and the compensator sums of its nrt row tiles are subtracted.
template <bool GRAD, int MIX = 1>
__device__ void finish_request(const Request &R, int nsum = -1) {
  constexpr int NV = GRAD ? 1 + num_grad(MIX) : 1;
  static_assert(NV <= kRedWidth, "reduction scratch too narrow");
  double *red3 = reduce_scratch();
  __shared__ int s_final;
  const SetView &S = R.set;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (blockDim.x + 31) >> 5;
  const unsigned parts = nsum >= 0 ? (unsigned)nsum : (unsigned)(S.nrt + comp_items(R));
  const int nrs = nsum >= 0 ? nsum : S.nrt;  // rt_sum slots
  __threadfence();
  __syncthreads();
  if (tid == 0) s_final = atomicAdd(R.rt_count + request_counters(R) - 1, 1u) == parts - 1u;
  __syncthreads();
  if (s_final) {
    __threadfence();
    // per thread, slots r = tid, tid + blockDim.x, ... in that order for every value q at once
    // (the loads of one slot issue together), then the warp tree and the warps in order
    double x[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) x[q] = 0.0;
    for (int r = tid; r < (nrs > S.nrt ? nrs : S.nrt); r += blockDim.x) {
      double a[NV], c[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        a[q] = r < nrs ? __ldcg(R.rt_sum + (size_t)r * kOut + q) : 0.0;
        c[q] = R.comp && r < S.nrt ? __ldcg(R.comp + (size_t)r * kOut + q) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        if (r < nrs) x[q] += a[q];
        if (R.comp && r < S.nrt) x[q] -= c[q];
      }
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x[q] += __shfl_down_sync(0xffffffffu, x[q], off);
      if (lane == 0) red3[warp * kRedWidth + q] = x[q];
    }
    __syncthreads();
    if (tid < NV) {
      double x = 0.0;
      for (int w = 0; w < nw; ++w) x += red3[w * kRedWidth + tid];
      // a sum that left the fixed-point range (red_fix) was not added: the results are NaN
      if (R.status && (__ldcg(R.status) & kStatusFixRange)) x = __longlong_as_double(0x7ff8000000000000ll);
      R.out[tid] = x;
    }
  }
  __syncthreads();
}

// Merge tree of a row tile's leaves (fused epilogue). An item enters at the node of its own
// leaves and climbs a binary tree over the tile's K leaves; at each node whose sibling subtree
// exists, the first CTA to arrive leaves its current sums in the slot of the node's first leaf
// and stops, and the second adds the sibling's sums to its own and climbs on. A node's value
// is left + right whichever side arrives second (floating-point addition commutes), so the
// sums do not depend on the order in which items finish. Returns true in the one CTA that
// completes the root: it then holds the tile's full row sums. store(slot) writes the CTA's
// current sums to a slot, merge(slot) adds a slot's sums to them (reading through L2). Called
// by every thread of the CTA. Returns 1 in the CTA that completes the root, 0 in a CTA that
// stopped at a node, -1 in a CTA that gave up waiting (the caller then calls mark_timeout for
// every request whose sums it carried). Two protocols, same sums:
//  - PUBLISH_FIRST: a CTA counts its arrival first; only the first stores (then adds a ready
//    mark), and the second waits for the mark if it is not there yet. The climbing CTA never
//    stores, which shortens the path of the last items (loglik + gradient: 24.6 KB slots).
//  - otherwise every arriving CTA stores before counting, so the second never waits (faster
//    for the 8 KB loglik slots, whose siblings tend to arrive close together).
// The wait is for a CTA that has already arrived and has nothing left to wait for, so it ends;
// it is still bounded (kMergeSpin polls and kMergeWaitNs of the global timer, whichever comes
// first), and a CTA that gives up sets kStatusMergeTimeout in the request's status word, which
// the host turns into HAWKES_E_DEVICE, writes NaN to the request's results and returns.
// With kFlagTestWithholdReady (tests only) the first CTA at each node of row tile 0 publishes its
// sums without the ready mark, so that its sibling's wait runs out.
// a node's counter: arrivals add 1 (at most 2, bits 0-1), the publisher's ready mark adds 4
constexpr unsigned kMergeArrived = 1u, kMergeReady = 4u;
constexpr int kMergeSpin = 1 << 22;
constexpr unsigned long long kMergeWaitNs = 500000000ull;  // 0.5 s

__device__ __forceinline__ unsigned load_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// A device wait of request R ran out: report it in R's status word and make its results NaN.
// Called by every thread of the CTA.
__device__ __forceinline__ void mark_timeout(const Request &R) {
  if (threadIdx.x == 0 && R.status) atomicOr(R.status, kStatusMergeTimeout);
  if (threadIdx.x < 7) R.out[threadIdx.x] = __longlong_as_double(0x7ff8000000000000ll);
}

template <bool PUBLISH_FIRST, class Store, class Merge>
__device__ int merge_tree(const Request &R, const PairItem &it, Store store, Merge merge) {
  __shared__ unsigned s_old, s_ok;
  const int K = R.slices;
  unsigned *cnt = R.rt_count + 2 * (size_t)it.rt * K;
  int node = it.node, width = it.span, off = 0;
  for (int w = 1; w < width; w <<= 1) off += (K + 2 * w - 1) / (2 * w);  // levels below the item
  while (width < K) {
    const int parent = node >> 1, sib = node ^ 1;
    if (sib * width < K) {  // the sibling subtree exists
      unsigned *c = cnt + off + parent;
      if (!PUBLISH_FIRST) {
        store(it.base + node * width / it.span);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_old = atomicAdd(c, kMergeArrived);
        __syncthreads();
        if (s_old == 0u) return 0;
        __threadfence();
        merge(it.base + sib * width / it.span);
        __syncthreads();
        off += (K + 2 * width - 1) / (2 * width);
        node = parent;
        width <<= 1;
        continue;
      }
      __syncthreads();
      if (threadIdx.x == 0) s_old = atomicAdd(c, kMergeArrived);
      __syncthreads();
      const unsigned old = s_old;
      if (old == 0u) {  // first: publish, then stop
        store(it.base + node * width / it.span);
        __threadfence();
        __syncthreads();
        const bool withhold = (R.flags & kFlagTestWithholdReady) && it.rt == 0;
        if (threadIdx.x == 0 && !withhold) atomicAdd(c, kMergeReady);
        return 0;
      }
      if (threadIdx.x == 0) {  // second: wait for the sibling's sums if they are not out yet
        bool ok = true;
        if (!(old & kMergeReady)) {
          const unsigned long long t0 = global_ns();
          for (int k = 0; !(load_acquire(c) & kMergeReady); ++k) {
            if (k >= kMergeSpin || global_ns() - t0 > kMergeWaitNs) {
              ok = false;
              break;
            }
            __nanosleep(64);
          }
        }
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) return -1;  // gave up waiting (never expected)
      __threadfence();
      merge(it.base + sib * width / it.span);
      __syncthreads();
    }
    off += (K + 2 * width - 1) / (2 * width);  // nodes at the parent's level
    node = parent;
    width <<= 1;
  }
  return 1;
}

// Log-intensity and gradient moments of event i from its row sums (Section 2.1, Eq. 1):
// lambda_i = A S_b + C S_s, v[0] += log lambda_i and, with GRAD, v[1..6] += (S_b, S_s, R_b,
// T_b, R_s, U_s) / lambda_i in stored units; also mu_i, xi_i and pi_i = xi_i / lambda_i of
// Eq. 2 when the request asks for them. Every gradient term (d lambda_i / d Theta) / lambda_i
// is a fixed linear combination of these six ratios, so rowtile_reduce applies the Theta
// factors once per row tile (grad_from_moments).
// With a two-component mixture (MIX = 2) the row sums carry S_s2 (and R_s2, U_s2) after the
// single-kernel ones, lambda_i = A S_b + C S_s1 + C_2 S_s2, and v[1 ..] takes all nine ratios.
// The natural log row_terms applies by default.
struct StdLog {
  __device__ __forceinline__ double operator()(double x) const { return log(x); }
};
// LogF: the log of lambda_i (StdLog, or the split epilogue's table log); FAST_RCP: 1 / lambda_i
// from the float32 reciprocal and one Newton step in float64 (relative error about 1e-14),
// 4 operations of the narrow float64 pipe instead of a division's 8 to 10.
template <bool GRAD, int MIX = 1, class LogF = StdLog, bool FAST_RCP = false>
__device__ __forceinline__ void row_terms(const Request &R, const MixConst &M2, int i, const double *sums, double *v,
                                          LogF logf = LogF()) {
  constexpr int NS = num_sums(GRAD, MIX);
  const double A = R.mu0 * R.k_ab, C = R.theta * R.k_cw;
  double xi = C * sums[1];
  if (MIX > 1) xi = fma(M2.theta2 * M2.k_cw2, sums[GRAD ? 6 : 2], xi);
  const double mu = A * sums[0], lam = mu + xi;
  if (R.mu_out) R.mu_out[i] = mu;
  if (R.xi_out) R.xi_out[i] = xi;
  if (R.pi_out) R.pi_out[i] = xi / lam;
  v[0] += logf(lam);
  if (GRAD) {
    double inv;
    if (FAST_RCP && lam > 1e-30 && lam < 1e30) {
      const double r0 = (double)__frcp_rn(__double2float_rn(lam));
      inv = fma(r0, fma(-lam, r0, 1.0), r0);
    } else {
      inv = 1.0 / lam;
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) v[1 + k] = fma(sums[k], inv, v[1 + k]);
  }
}

// The six gradient terms of Eq. 1's log-intensity sum from the moment ratios m = (sum_i
// S_b/lambda_i, S_s/lambda, R_b/lambda, T_b/lambda, R_s/lambda, U_s/lambda) of row_terms:
//   d/d mu0    = k_ab m_Sb
//   d/d tau_x  = A/tau_x (-2 m_Sb + m_Rb / tau_x^2)
//   d/d tau_t  = A/tau_t (-m_Sb + m_Tb / tau_t^2)        (m_Tb, m_Us rescaled by tscale)
//   d/d theta  = k_cw m_Ss
//   d/d omega  = C (m_Ss / omega - m_Us)
//   d/d h      = C/h (-2 m_Ss + m_Rs / h^2)
// (component 2 of a mixture, from m[6..8] = S_s2, R_s2, U_s2 ratios: the same three formulas with
// theta_2, omega_2, h_2 into g[6..8]).
template <int MIX = 1>
__device__ __forceinline__ void grad_from_moments(const Request &R, const MixConst &M2, const double *m, double *g) {
  const double A = R.mu0 * R.k_ab, C = R.theta * R.k_cw;
  const double itx = R.inv_tx, itt = R.inv_tt, ih = R.inv_h, iom = R.inv_om;
  const double Sb = m[0], Ss = m[1], Rb = m[2], Tb = m[3] * R.tscale * R.tscale, Rs = m[4], Us = m[5] * R.tscale;
  g[0] = R.k_ab * Sb;
  g[1] = A * itx * (-2.0 * Sb + Rb * itx * itx);
  g[2] = A * itt * (-Sb + Tb * itt * itt);
  g[3] = R.k_cw * Ss;
  g[4] = C * (Ss * iom - Us);
  g[5] = C * ih * (-2.0 * Ss + Rs * ih * ih);
  if (MIX > 1) {
    const double C2 = M2.theta2 * M2.k_cw2, ih2 = M2.inv_h2;
    const double Ss2 = m[6], Rs2 = m[7], Us2 = m[8] * R.tscale;
    g[6] = M2.k_cw2 * Ss2;
    g[7] = C2 * (Ss2 * M2.inv_om2 - Us2);
    g[8] = C2 * ih2 * (-2.0 * Ss2 + Rs2 * ih2 * ih2);
  }
}

// End of row tile rt's epilogue: sum every thread's row terms v in a fixed order (warp tree,
// warps in order), turn the moment ratios into gradient terms (grad_from_moments), store
// them in R.rt_sum, then finish_request. Called by every thread of the CTA.
template <bool GRAD, int MIX = 1, bool FINISH = true>
__device__ void rowtile_reduce(const Request &R, const MixConst &M2, int rt, const double *v) {
  constexpr int NV = GRAD ? 1 + num_sums(true, MIX) : 1;  // log lambda and the moment ratios
  static_assert(NV <= kRedWidth, "reduction scratch too narrow");
  double *red2 = reduce_scratch(), *tot = red2 + kMaxCtaWarps * kRedWidth;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();  // the scratch's previous use is over
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double x = v[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if (lane == 0) red2[warp * kRedWidth + q] = x;
  }
  __syncthreads();
  if (tid < NV) {
    double x = 0.0;
    for (int w = 0; w < nw; ++w) x += red2[w * kRedWidth + tid];
    tot[tid] = x;
  }
  __syncthreads();
  if (tid == 0) {
    R.rt_sum[(size_t)rt * kOut] = tot[0];
    if (GRAD) {
      double g[num_grad(MIX)];
      grad_from_moments<MIX>(R, M2, tot + 1, g);
#pragma unroll
      for (int k = 0; k < num_grad(MIX); ++k) R.rt_sum[(size_t)rt * kOut + 1 + k] = g[k];
    }
  }
  if (FINISH) finish_request<GRAD, MIX>(R);
}
#endif

}  // namespace hk
