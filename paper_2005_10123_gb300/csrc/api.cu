// Host runtime behind include/hawkes.h: contexts, resident event sets, synchronous and
// batched evaluation, and the serving queue.
//
// Every evaluation is one "batch" launch on a stream (after one memset of its counters): the
// pair kernel (mixed, fp64, or the grouped mixed kernel for several parameter vectors on one
// set) runs one CTA per work item, merges each row tile's partial sums in a fixed tree and
// finishes every row tile and request itself (log lambda_n - Lambda_n, gradient terms, fixed-
// order reductions). Outside the grouped kernel a request's arithmetic depends only on its own
// set, parameters and work decomposition, never on the other requests of its batch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/hawkes.h"
#include "upload.h"

using namespace hk;

namespace {

constexpr int kKinds = 3;  // kernel kinds: 0 mixed loglik, 1 mixed grad, 2 fp64
constexpr int kFlights = 3;  // serving launches in flight at once
constexpr double kLog2e = 1.4426950408889634074;

int kind_of(int mode, int grad) { return mode == HAWKES_MIXED ? (grad ? 1 : 0) : 2; }
// Pair sums per event of a request with m trigger components (partial-sum slot width / kRowTile).
int sums_of(int grad, int m = 1) { return num_sums(grad != 0, m); }

struct EventSetRec {
  int32_t id = 0;
  int64_t n = 0, npad = 0;
  int nrt = 0, nct = 0;
  void *dev = nullptr;  // one allocation for coordinates and tie indices
  size_t bytes = 0;
  float *x32 = nullptr, *y32 = nullptr, *t32 = nullptr;
  double *x64 = nullptr, *y64 = nullptr, *t64 = nullptr;
  int *lo32 = nullptr, *lo64 = nullptr;
  double t_first32 = 0, t_last32 = 0, t_first64 = 0, t_last64 = 0;
  WinTable win32{}, win64{};  // column-tile lookups (device pointers)
  int slices[kKinds] = {1, 1, 1};  // slices per row tile, per kernel kind
  int refs = 0;  // queued or running serving requests
  bool released = false;
};

struct Workspace {
  void *dev = nullptr;
  size_t bytes = 0;
};

struct TicketRec {
  int32_t set_id = 0;
  hawkes_params p{};
  int grad = 0, mode = 0, flags = 0;
  int status = HAWKES_E_PENDING;
  bool done = false;
  double ll = 0, g[6] = {0, 0, 0, 0, 0, 0};
  size_t footprint = 0;
  int64_t t_submit = 0, t_launch = 0, t_done = 0;  // steady-clock nanoseconds
};

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Flight {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<uint64_t> ids;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  double *host_out = nullptr;  // pinned, kFixedBytes: status words, then kMaxBatch * kOut results
  std::vector<EventSetRec *> sets;
};

}  // namespace

struct hawkes_ctx {
  int device = 0;
  int sms = 0;
  int host_direct = 0;  // the device reads pageable host memory (uploads skip the copy)
  int occ[kKinds] = {1, 1, 1};
  int occ_launch[2][2] = {{1, 1}, {1, 1}};  // [mode][grad]
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;
  std::atomic<size_t> used{0};
  int flags = 0;
  std::mutex mu;  // sets, sync workspace, synchronous calls
  std::map<int32_t, EventSetRec *> sets;
  int32_t next_set = 1;
  Workspace sync_ws;
  double *pinned_out = nullptr;  // kFixedBytes: status words, then kMaxBatch * kOut results
  cudaMemPool_t pool = nullptr;   // device memory of event sets and serving workspaces (stream-ordered)
  char *stage = nullptr;          // pinned host word for the upload checks (guarded by mu)
  char *bounce = nullptr;         // pinned bounce buffer for per-event rows (guarded by mu)
  cudaEvent_t bounce_ev[2] = {nullptr, nullptr};
  // hawkes_set_kernel_timing: events around the pair kernel and the split epilogue of every
  // evaluation on the context's own stream (kev[0] before, kev[1] between, kev[2] after)
  int ktime = 0;
  cudaEvent_t kev[3] = {nullptr, nullptr, nullptr};
  int kev_recorded = 0;
  cudaStream_t copy_stream = nullptr;  // copies out of pi batches, beside the launches
  std::vector<cudaEvent_t> chunk_ev;   // one per launch of a pi batch
  std::string last_cuda;
  // serving
  std::mutex smu;
  std::condition_variable scv;   // scheduler wake-ups
  std::condition_variable done_cv;  // ticket completions
  std::unordered_map<uint64_t, TicketRec> tickets;
  std::deque<uint64_t> pending;
  uint64_t next_ticket = 1;
  Flight flights[kFlights];
  bool flights_ready = false;
  std::thread sched_thread;
  bool sched_running = false;
  bool shutdown = false;
  int64_t n_submitted = 0, n_completed = 0, n_failed = 0, n_launches = 0;
  size_t serving_bytes = 0;
};

namespace {

int cuda_fail(hawkes_ctx *ctx, cudaError_t e) {
  if (ctx) ctx->last_cuda = cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return HAWKES_E_NOMEM;
  return HAWKES_E_CUDA;
}

#define HK_CUDA(ctx, call)                         \
  do {                                             \
    cudaError_t _e = (call);                       \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e); \
  } while (0)

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

int check_params(const hawkes_params *p) {
  if (!p) return HAWKES_E_INVAL;
  if (!finite_pos(p->mu0) || !finite_pos(p->tau_x) || !finite_pos(p->tau_t) || !finite_pos(p->omega) ||
      !finite_pos(p->h))
    return HAWKES_E_INVAL;
  if (!std::isfinite(p->theta) || p->theta < 0.0) return HAWKES_E_INVAL;
  return HAWKES_OK;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Leaves per row tile for a kernel kind: about kItemsPerSlot items per resident CTA, at most
// one column tile per leaf. The mixed kernels cut twice as fine: their items span 4, 2 or 1
// leaves along the launch order (launch_tiers).
#ifndef HK_ITEMS_PER_SLOT
#define HK_ITEMS_PER_SLOT 3  // 85k loglik+grad: 3 0.363 ms, 4 0.371 ms, 2 0.366 ms (same box)
#endif
// Smallest mixed-precision batch run by the grouped kernel; smaller batches run as independent
// requests in one launch, each with the shared background, which was faster below these sizes
// (N = 85,000: 2 requests 0.89 against 1.00 ms, 8 requests 3.19 against 3.35 ms, 16 requests
// 6.55 against 6.41 ms with the gradient; sets of 8,000 and 20,000 events cross over between 8
// and 16).
#ifndef HK_GROUP_MIN_K
#define HK_GROUP_MIN_K 12  // loglik + gradient
#endif
#ifndef HK_GROUP_MIN_K_LL
#define HK_GROUP_MIN_K_LL 16  // loglik only
#endif
constexpr int kItemsPerSlot = HK_ITEMS_PER_SLOT;
#ifndef HK_TIER_WIDE_PCT
#define HK_TIER_WIDE_PCT 50  // percent of the row tiles (launched first) with 4-leaf items
#endif
#ifndef HK_TIER_FINE_PCT
#define HK_TIER_FINE_PCT 25  // percent of the row tiles (launched last) with 1-leaf items
#endif
int slices_for(int nrt, int nct, int resident_ctas, bool tiered) {
  const int want = (kItemsPerSlot * resident_ctas + nrt - 1) / nrt * (tiered ? 2 : 1);
  return std::max(1, std::min(want, nct));
}

// Item spans along the launch order (see Request). The mixed kernel: the first half of the
// row tiles take 4-leaf items, the next quarter 2-leaf items and the last quarter 1-leaf items,
// so the launch ends on short items. The grouped kernel, whose items already carry several
// requests, runs 2-leaf items throughout (measured faster for it); the float64 kernel 1-leaf.
void launch_tiers(int nrt, int mode, bool grouped, int *wide, int *coarse) {
  if (mode != HAWKES_MIXED) {
    *wide = *coarse = 0;
  } else if (grouped) {
    *wide = 0;
    *coarse = nrt;
  } else {
    *wide = nrt * HK_TIER_WIDE_PCT / 100;
    *coarse = nrt - nrt * HK_TIER_FINE_PCT / 100;
  }
}

// Reaches (days) of Section 2.1's pair terms: past bg of |t_n - t_n'| a background term, past
// trig of t_n - t_n' a trigger term contributes nothing at the working precision.
// - float32 (mixed) with the self term in the background sum (the default): lambda_n >= A (see
//   below). A background term is e_b = 2^-q with q >= dt'^2, dt' = beta dt; past q = Q,
//   Q = log2 N + 40, it is below 2^-40 / N, and all N of a row together stay below 2^-40 of
//   lambda_n (2^-16 of float32's rounding unit). A trigger term of weight C (below) past
//   omega dt log2(e) = Q + log2(C / A) (when C > A) likewise. Both exponents stop at the point
//   where ex2.approx.ftz returns +0 (q = 130 and 131), which is where the reaches stand without
//   the floor: with HAWKES_FLAG_EXCLUDE_SELF or HAWKES_FLAG_DENSE every term that is not exactly
//   zero in float32 is kept.
// - float64 with the self term in the background sum (the default): S_b >= 1, so lambda_n >= A
//   = mu0 / ((2 pi)^(3/2) tau_x^2 tau_t). A background term beyond dt^2 / (2 tau_t^2) = E,
//   E = ln N + 70 ln 2, is below e^-E, and all N of a row together stay below 2^-70 of
//   lambda_n (1/128 of float64's rounding unit); a trigger term of weight C = theta omega /
//   (2 pi h^2) beyond omega dt = E + ln(C / A) (when C > A) likewise. The sums are those of
//   every pair up to float64 rounding, and the window is a third to a quarter as long.
// - float64 without that floor (HAWKES_FLAG_EXCLUDE_SELF, where S_b can be as small as one
//   term), or with HAWKES_FLAG_DENSE (every pair): exp returns +0 far below -745, so both
//   exponents go to 805.
void term_reaches(const hawkes_params *p, int mode, float beta32, int flags, int64_t n, double *bg, double *trig) {
  if (mode == HAWKES_MIXED) {
    double qb = 130.0, qt = 131.0;
    if (!(flags & (HAWKES_FLAG_EXCLUDE_SELF | HAWKES_FLAG_DENSE))) {
      const double two_pi = 6.28318530717958647693;
      const double A = p->mu0 / (two_pi * std::sqrt(two_pi) * p->tau_x * p->tau_x * p->tau_t);
      const double C = p->theta * p->omega / (two_pi * p->h * p->h);
      const double Q = std::log2((double)std::max<int64_t>(n, 1)) + 40.0;
      qb = std::min(qb, Q);
      qt = std::min(qt, Q + (C > A ? std::log2(C / A) : 0.0));
    }
    *bg = std::sqrt(qb) / (double)beta32;
    *trig = qt / (p->omega * kLog2e);
  } else if (!(flags & (HAWKES_FLAG_EXCLUDE_SELF | HAWKES_FLAG_DENSE))) {
    const double two_pi = 6.28318530717958647693;
    const double A = p->mu0 / (two_pi * std::sqrt(two_pi) * p->tau_x * p->tau_x * p->tau_t);
    const double C = p->theta * p->omega / (two_pi * p->h * p->h);
    const double E = std::log((double)std::max<int64_t>(n, 1)) + 70.0 * std::log(2.0);
    *bg = std::sqrt(E * 2.0) * p->tau_t;
    *trig = (E + (C > A ? std::log(C / A) : 0.0)) / p->omega;
  } else {
    *bg = std::sqrt(805.0 * 2.0) * p->tau_t;
    *trig = 805.0 / p->omega;
  }
}

// The column windows' cut-offs: the reaches with one percent of margin for the rounding of the
// time differences. Columns earlier than a row carry both terms, later ones the background only.
void exact_zero_cutoffs(const hawkes_params *p, int mode, float beta32, int flags, int64_t n, double *early,
                        double *late, double *trig_out = nullptr) {
  double bg, trig;
  term_reaches(p, mode, beta32, flags, n, &bg, &trig);
  bg *= 1.01;
  trig *= 1.01;
  *early = std::max(bg, trig);
  *late = bg;
  if (trig_out) *trig_out = trig;
}

// Whether a request on S shares the background terms of far column tiles (see SymPlan in
// hk_internal.h): mixed precision, a time table, and none of the flags that ask for row-by-row
// evaluation (exclude-self makes lambda_n's background sum unbounded below, which the fixed-point
// column sums would not resolve; dense and no-symmetry ask for every ordered pair).
// The test flag that withholds a merge-tree ready mark asks for the merge tree, which the shared
// background does not use.
bool use_symmetry(const EventSetRec *S, int mode, int flags) {
  return mode == HAWKES_MIXED && S->win32.nb > 0 &&
         !(flags & (HAWKES_FLAG_EXCLUDE_SELF | HAWKES_FLAG_DENSE | HAWKES_FLAG_NO_SYMMETRY | kFlagTestWithholdReady));
}

// Float64 constants of the epilogue and compensator, from Theta (Section 2.1, d = 2).
void set_epilogue_constants(Request *R) {
  const double two_pi = 6.28318530717958647693;
  R->k_ab = 1.0 / (two_pi * std::sqrt(two_pi) * R->tau_x * R->tau_x * R->tau_t);
  R->k_cw = R->omega / (two_pi * R->h * R->h);
  R->inv_tx = 1.0 / R->tau_x;
  R->inv_tt = 1.0 / R->tau_t;
  R->inv_h = 1.0 / R->h;
  R->inv_om = 1.0 / R->omega;
}

// Request descriptor for one evaluation of set `S` at Theta `p`.
int make_request(hawkes_ctx *ctx, const EventSetRec *S, const hawkes_params *p, int mode, int grad,
                 int flags, Request *R) {
  std::memset(R, 0, sizeof(*R));
  R->set.x32 = S->x32; R->set.y32 = S->y32; R->set.t32 = S->t32;
  R->set.x64 = S->x64; R->set.y64 = S->y64; R->set.t64 = S->t64;
  R->set.lo32 = S->lo32; R->set.lo64 = S->lo64;
  R->set.win32 = S->win32; R->set.win64 = S->win64;
  R->set.n = (int)S->n; R->set.npad = (int)S->npad; R->set.nrt = S->nrt; R->set.nct = S->nct;
  R->slices = S->slices[kind_of(mode, grad)];
  launch_tiers(S->nrt, mode, false, &R->wide, &R->coarse);
  R->grad = grad;
  R->flags = flags;
  set_mixed_constants(R, p->tau_x, p->tau_t, p->omega, p->h);
  R->da = 1.0 / (2.0 * p->tau_x * p->tau_x);
  R->db = 1.0 / (2.0 * p->tau_t * p->tau_t);
  R->dc = 1.0 / (2.0 * p->h * p->h);
  R->mu0 = p->mu0; R->tau_x = p->tau_x; R->tau_t = p->tau_t;
  R->theta = p->theta; R->omega = p->omega; R->h = p->h;
  set_epilogue_constants(R);
  if (mode == HAWKES_MIXED) {
    // the float32 path must keep every scaled quantity finite and below the padding value
    const double span = (S->t_last32 - S->t_first32) * (double)R->beta;
    if (!(R->a2 > 0.f) || !(R->beta > 0.f) || !(R->b2 > 0.f) || !(R->s_hi > 0.f) || !std::isfinite(R->wn) ||
        !(R->cn < 0.f) || !std::isfinite(R->a2) || !std::isfinite(R->b2) || !std::isfinite(R->cn) || span > 1.0e15)
      return HAWKES_E_INVAL;
    R->t_last = S->t_last32;
  } else {
    R->t_last = S->t_last64;
    R->tscale = 1.0;
  }
  exact_zero_cutoffs(p, mode, R->beta, flags, S->n, &R->cut_early, &R->cut_late, &R->trig_cut);
  R->sym = use_symmetry(S, mode, flags) ? (HK_SYM_NEAR ? 2 : 1) : 0;
  R->mix = 1;
  set_fix_bits(R, grad, 1, p->h, p->omega, 0.0, 0.0, S->t_last32 - S->t_first32);
  (void)ctx;
  return HAWKES_OK;
}

// Component 2 of a trigger mixture (the Discussion's extension; hawkes_loglik_mix): the second
// triggering function's constants go to the launch (Batch::mix2), and the exact-zero windows take
// the longer of the two trigger reaches. R holds the request made from component 1.
int set_mixture(const hawkes_mix_params *m, int mode, double span, Request *R, MixConst *M2) {
  const double log2e = kLog2e, th2 = m->theta[1], om2 = m->omega[1], h2 = m->h[1];
  if (!std::isfinite(th2) || th2 < 0.0 || !finite_pos(om2) || !finite_pos(h2)) return HAWKES_E_INVAL;
  std::memset(M2, 0, sizeof(*M2));
  M2->theta2 = th2;
  M2->omega2 = om2;
  M2->h2 = h2;
  M2->dc2 = 1.0 / (2.0 * h2 * h2);
  M2->k_cw2 = om2 / (6.28318530717958647693 * h2 * h2);
  M2->inv_h2 = 1.0 / h2;
  M2->inv_om2 = 1.0 / om2;
  M2->wn2 = (float)(-om2 * log2e / (1.0 / R->tscale));
  M2->cn2 = (float)(-log2e / (2.0 * h2 * h2));
  if (mode == HAWKES_FP64) M2->wn2 = 0.f;  // the float64 kernel uses omega2 and dc2
  else if (!std::isfinite(M2->wn2) || !(M2->cn2 < 0.f) || !std::isfinite(M2->cn2)) return HAWKES_E_INVAL;
  hawkes_params p2{R->mu0, R->tau_x, R->tau_t, th2, om2, h2};
  double early2, late2, trig2;
  exact_zero_cutoffs(&p2, mode, R->beta, R->flags, R->set.n, &early2, &late2, &trig2);
  R->trig_cut = std::max(R->trig_cut, trig2);
  R->cut_early = std::max(R->cut_early, early2);
  R->mix = 2;
  set_fix_bits(R, R->grad, 2, R->h, R->omega, h2, om2, span);
  return HAWKES_OK;
}

// Device bytes one request needs: partial sums, compensator sums, row-tile sums.
// Partial-sum slots of one request on S: its pair items, alone or grouped (see Request).
size_t set_slots(const EventSetRec *S, int mode, int grad) {
  Request R;
  std::memset(&R, 0, sizeof(R));
  R.set.nrt = S->nrt;
  R.slices = S->slices[kind_of(mode, grad)];
  launch_tiers(S->nrt, mode, false, &R.wide, &R.coarse);
  const int alone = pair_items(R);
  launch_tiers(S->nrt, mode, true, &R.wide, &R.coarse);
  return (size_t)std::max(alone, pair_items(R));
}

// With the shared background (sym) a request keeps no partial-sum slots: its per-event sums sit
// in fixed point among its counters (counter_bytes).
size_t request_footprint(const EventSetRec *S, int mode, int grad, int m = 1, int sym = 0) {
  const size_t items = sym ? 0 : set_slots(S, mode, grad);
  size_t b = align_up(items * sums_of(grad, m) * kRowTile * sizeof(double), 256);
  b += 4 * align_up((size_t)S->nrt * kOut * sizeof(double), 256);  // comp, rt_sum (3 nrt slots)
  return b;
}

// Bytes of a request's counters, kept in one zeroed region per batch: the merge-tree nodes of
// its row tiles and one final counter (Request::rt_count); with sym, the row tiles' completion
// counters (Request::rt_done) and the per-event fixed-point sums (Request::fixsum, num_sums x
// npad integers: 4.1 MB for loglik + gradient at N = 85,000).
size_t merge_counter_bytes(const EventSetRec *S, int mode, int grad) {
  return (2 * (size_t)S->nrt * S->slices[kind_of(mode, grad)] + 1) * sizeof(unsigned);
}
size_t counter_bytes(const EventSetRec *S, int mode, int grad, int sym, int m = 1) {
  size_t b = merge_counter_bytes(S, mode, grad);
  if (sym) b = align_up(b + (size_t)S->nrt * sizeof(unsigned), 256) + (size_t)num_sums(grad != 0, m) * S->npad * 8;
  return align_up(b, 256);
}

// Batch workspace: a 256-byte header holding one device status word per request (see
// Request::status), the per-request outputs (8 doubles each), then every request's completion
// counters. One memset of these (kFixedBytes + the batch's counter bytes) zeroes everything
// that must start at 0; one copy of the first kHdrBytes + 64 k bytes brings the status words
// and results back.
constexpr size_t kHdrBytes = 256;
constexpr size_t kOutBytes = (size_t)kMaxBatch * kOut * sizeof(double);
constexpr size_t kFixedBytes = kHdrBytes + kOutBytes;
static_assert(kHdrBytes >= kMaxBatch * sizeof(unsigned), "one status word per request");

// The status of request r from the copied-back header: HAWKES_E_DEVICE if one of its device
// waits ran out (its results are NaN), else HAWKES_OK (a sum outside the fixed-point range,
// kStatusFixRange, leaves NaN results with HAWKES_OK, as any non-finite evaluation does).
int device_status(const void *header, int r) {
  return (((const unsigned *)header)[r] & kStatusMergeTimeout) ? HAWKES_E_DEVICE : HAWKES_OK;
}

// Carve one request's workspace out of `base` (as sized by request_footprint with the same m and
// fix) and its counters out of `counters` (as sized by counter_bytes). fix: the request adds its
// sums in fixed point (Request::fixsum), with the shared background or in a grouped batch.
void bind_workspace(Request *R, const EventSetRec *S, int mode, int grad, char *base, double *out,
                    unsigned *counters, int m, int fix) {
  if (fix) {
    const size_t m = merge_counter_bytes(S, mode, grad);
    R->rt_done = (unsigned *)((char *)counters + m);
    R->fixsum = (long long *)((char *)counters + align_up(m + (size_t)S->nrt * sizeof(unsigned), 256));
  }
  const size_t items = fix ? 0 : set_slots(S, mode, grad);
  size_t off = 0;
  R->partials = (double *)(base + off);
  off += align_up(items * sums_of(grad, m) * kRowTile * sizeof(double), 256);
  R->comp = (double *)(base + off);
  off += align_up((size_t)S->nrt * kOut * sizeof(double), 256);
  R->rt_sum = (double *)(base + off);
  R->rt_count = counters;
  R->out = out;
}

// Enqueue the pair kernel (one CTA per item) for a prepared batch on `s`; it finishes every
// row tile and every request itself (fused epilogue), except, in mixed precision, the requests
// with the shared background, whose epilogues run in a second launch on the same stream
// (launch_epilogue_fix). Every request's completion counters must already be zero (the caller
// clears them with one memset).
int launch_batch(hawkes_ctx *ctx, Batch &b, int mode, int grad, cudaStream_t s) {
  b.mode = mode == HAWKES_MIXED ? 1 : 0;
  b.fused = 1;
  b.split = mode == HAWKES_MIXED && !b.group ? 1 : 0;
  long long items = 0;
  if (b.group) {  // grouped kernel: every request's compensator items, then the groups' pair items
    const int G = b.group;
    for (int r = 0; r < b.nreq; ++r) items += comp_items(b.req[r]);
    b.comp_total = (int)items;
    items += (long long)((b.nreq + G - 1) / G) * pair_items(b.req[0]);
  } else {
    for (int r = 0; r < b.nreq; ++r) {
      b.req[r].item_begin = (int)items;
      items += request_items(b.req[r]);
    }
  }
  if (items > 0x7fffffffLL) return HAWKES_E_INVAL;
  for (int r = 0; r < b.nreq; ++r)  // a sym request's row sums are finished by the split epilogue
    if (b.req[r].sym && !b.split) return HAWKES_E_INVAL;
  b.total_items = (int)items;
  const bool timed = ctx->ktime && s == ctx->stream;
  if (timed) HK_CUDA(ctx, cudaEventRecord(ctx->kev[0], s));
  if (b.group) HK_CUDA(ctx, launch_pair_group(b, grad != 0, s));
  else if (mode == HAWKES_MIXED) HK_CUDA(ctx, launch_pair_mixed(b, grad != 0, s));
  else HK_CUDA(ctx, launch_pair_fp64(b, grad != 0, s));
  if (timed) HK_CUDA(ctx, cudaEventRecord(ctx->kev[1], s));
  if (!b.group && mode == HAWKES_MIXED) HK_CUDA(ctx, launch_epilogue_fix(b, grad != 0, s));
  if (timed) {
    HK_CUDA(ctx, cudaEventRecord(ctx->kev[2], s));
    ctx->kev_recorded = 1;
  }
  return HAWKES_OK;
}

int ensure_sync_ws(hawkes_ctx *ctx, size_t need) {
  if (ctx->sync_ws.bytes >= need) return HAWKES_OK;
  need = align_up(need + need / 4, 1 << 20);
  const size_t old = ctx->sync_ws.bytes;
  if (ctx->used.load() - old + need > ctx->budget) return HAWKES_E_ADMISSION;
  if (ctx->sync_ws.dev) {
    HK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->sync_ws.dev);
    ctx->sync_ws.dev = nullptr;
    ctx->used -= old;
    ctx->sync_ws.bytes = 0;
  }
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, need);
  if (e != cudaSuccess) return cuda_fail(ctx, e);
  ctx->sync_ws.dev = p;
  ctx->sync_ws.bytes = need;
  ctx->used += need;
  return HAWKES_OK;
}

EventSetRec *find_set(hawkes_ctx *ctx, int32_t id) {
  auto it = ctx->sets.find(id);
  if (it == ctx->sets.end() || it->second->released) return nullptr;
  return it->second;
}

void free_set(hawkes_ctx *ctx, EventSetRec *S) {
  // stream-ordered: after the work already queued on the context's stream, the last user of a
  // set outside serving (serving requests hold a reference until their launch has finished)
  if (S->dev) cudaFreeAsync(S->dev, ctx->stream);
  ctx->used -= S->bytes;
  delete S;
}

// Device rows (n doubles each) to caller-owned host memory through a pinned bounce buffer
// in two halves: the device-to-host copy into one half overlaps the host copy out of the
// other. Direct copies into pageable memory ran at about 2 GB/s on the Grace host. Called
// with ctx->mu held; the copies are issued on ctx->stream after the work that writes `src`.
constexpr size_t kBounceHalf = (size_t)4 << 20;
int rows_to_host(hawkes_ctx *ctx, double *const *dst, const char *const *src, int rows, size_t nb,
                 cudaStream_t stream) {
  if (!ctx->bounce) {
    HK_CUDA(ctx, cudaMallocHost((void **)&ctx->bounce, 2 * kBounceHalf));
    for (cudaEvent_t &ev : ctx->bounce_ev) HK_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  struct Piece { char *dst; size_t len; };
  std::vector<Piece> pend[2];
  size_t fill[2] = {0, 0};
  int h = 0;
  auto drain = [&](int w) -> int {
    if (pend[w].empty()) return HAWKES_OK;
    HK_CUDA(ctx, cudaEventSynchronize(ctx->bounce_ev[w]));
    size_t off = 0;
    for (const Piece &p : pend[w]) {
      std::memcpy(p.dst, ctx->bounce + (size_t)w * kBounceHalf + off, p.len);
      off += p.len;
    }
    pend[w].clear();
    fill[w] = 0;
    return HAWKES_OK;
  };
  for (int r = 0; r < rows; ++r)
    for (size_t o = 0; o < nb; o += kBounceHalf) {
      const size_t len = std::min(kBounceHalf, nb - o);
      if (fill[h] + len > kBounceHalf) {  // this half is full: hand it over, take the other
        HK_CUDA(ctx, cudaEventRecord(ctx->bounce_ev[h], stream));
        h ^= 1;
        if (int rc = drain(h)) return rc;
      }
      HK_CUDA(ctx, cudaMemcpyAsync(ctx->bounce + (size_t)h * kBounceHalf + fill[h], src[r] + o, len,
                                   cudaMemcpyDeviceToHost, stream));
      pend[h].push_back(Piece{(char *)dst[r] + o, len});
      fill[h] += len;
    }
  HK_CUDA(ctx, cudaEventRecord(ctx->bounce_ev[h], stream));
  if (int rc = drain(h ^ 1)) return rc;
  return drain(h);
}

// Synchronous evaluation of k requests on one set (k = 1 for the single calls).
// Results (ell and the gradient per request) land in host_out[kOut * r]; device_out, if given
// (k = 1 only), receives them on the device instead and the call does not block.
// mu_out / xi_out (k = 1) receive the per-event mu_n and xi_n of Eq. 2, pi_out (k rows of n)
// the per-event pi_n of every request.
// eval_sync with ctx->mu held and the set found. pi_dev (device, rows of row_bytes for each
// parameter vector) receives pi instead of pi_out when given; with device_out the call
// returns once the launch is enqueued.
// mix (k = 1 only): a two-component trigger mixture; params[0] then holds its component 1.
int eval_locked(hawkes_ctx *ctx, EventSetRec *S, int k, const hawkes_params *params, int mode, int grad,
                double *host_out, double *device_out, double *mu_out, double *xi_out, double *pi_out,
                char *pi_dev, const hawkes_mix_params *mix = nullptr);

int eval_sync(hawkes_ctx *ctx, int32_t set_id, int k, const hawkes_params *params, int mode, int grad,
              double *host_out, double *device_out, double *mu_out, double *xi_out, double *pi_out,
              const hawkes_mix_params *mix = nullptr) {
  if (mode != HAWKES_FP64 && mode != HAWKES_MIXED) return HAWKES_E_INVAL;
  if (k < 1 || k > kMaxBatch) return HAWKES_E_INVAL;
  for (int r = 0; r < k; ++r)
    if (int rc = check_params(&params[r])) return rc;
  std::lock_guard<std::mutex> lock(ctx->mu);
  EventSetRec *S = find_set(ctx, set_id);
  if (!S) return HAWKES_E_NOSET;
  return eval_locked(ctx, S, k, params, mode, grad, host_out, device_out, mu_out, xi_out, pi_out, nullptr, mix);
}

int eval_locked(hawkes_ctx *ctx, EventSetRec *S, int k, const hawkes_params *params, int mode, int grad,
                double *host_out, double *device_out, double *mu_out, double *xi_out, double *pi_out,
                char *pi_dev, const hawkes_mix_params *mix) {
  if (mix && k != 1) return HAWKES_E_INVAL;
  const int m = mix ? 2 : 1;  // trigger components
  // per-event rows. mu and xi (one request) are written by the kernel straight into the
  // caller's host arrays where the device writes pageable host memory (0.50 -> 0.40 ms at
  // 85k). pi rows (k requests) are staged in device memory and copied out through the bounce
  // buffer: written in place they were slower (85 against 69 ms for 256 x 85k), the host
  // faulting in the caller's fresh pages one by one.
  const bool direct_rows = ctx->host_direct != 0;
  const size_t row_bytes = align_up((size_t)S->n * sizeof(double), 256);
  const size_t rows_bytes =
      ((mu_out || xi_out) && !direct_rows ? 2 * row_bytes : 0) + (pi_out && !pi_dev ? (size_t)k * row_bytes : 0);
  // From HK_GROUP_MIN_K (gradient) or HK_GROUP_MIN_K_LL mixed-precision requests on this set,
  // groups of group_size(grad, k) share each pair's geometry (grouped kernel, moments in raw
  // units). Groups are consecutive requests in order of tau_t, so a group's members have
  // similar column windows; request r of the launch is params[order[r]] and writes its
  // results to that parameter vector's place. The other launches run each request as it runs
  // alone, sharing the background terms of far column tiles where use_symmetry allows it.
  const bool grouped = k >= (grad ? HK_GROUP_MIN_K : HK_GROUP_MIN_K_LL) && mode == HAWKES_MIXED;
  const int sym = !grouped && use_symmetry(S, mode, ctx->flags) ? 1 : 0;
  // grouped batches add their sums in fixed point too, unless exclude-self takes away the
  // background sum's floor of 1 or the test flag asks for the merge tree
  const int gfix = grouped && !(ctx->flags & (HAWKES_FLAG_EXCLUDE_SELF | kFlagTestWithholdReady)) ? 1 : 0;
  const int fix = sym || gfix;
  const size_t per = request_footprint(S, mode, grad, m, fix);
  const size_t cnt_one = counter_bytes(S, mode, grad, fix, m);
  const size_t cnt = align_up(cnt_one * k, 256);
  const size_t need = kFixedBytes + cnt + rows_bytes + per * k;
  if (int rc = ensure_sync_ws(ctx, need)) return rc;
  char *base = (char *)ctx->sync_ws.dev;
  std::unique_ptr<Batch> b(new Batch());
  std::memset(b.get(), 0, sizeof(Batch));
  b->nreq = k;
  double *outs = (double *)(base + kHdrBytes);
  char *cnt_base = base + kFixedBytes;
  char *rows_base = cnt_base + cnt;
  char *req_base = rows_base + rows_bytes;
  int order[kMaxBatch];
  for (int r = 0; r < k; ++r) order[r] = r;
  if (grouped)
    std::stable_sort(order, order + k, [&](int a, int c) { return params[a].tau_t < params[c].tau_t; });
  for (int r = 0; r < k; ++r) {
    const int q = order[r];
    if (int rc = make_request(ctx, S, &params[q], mode, grad, ctx->flags, &b->req[r])) return rc;
    if (!sym) b->req[r].sym = 0;  // grouped (make_request chose the level otherwise)
    if (mix)
      if (int rc = set_mixture(mix, mode, S->t_last32 - S->t_first32, &b->req[r], &b->mix2)) return rc;
    bind_workspace(&b->req[r], S, mode, grad, req_base + (size_t)r * per,
                   device_out ? device_out + kOut * q : outs + kOut * q, (unsigned *)(cnt_base + (size_t)r * cnt_one),
                   m, fix);
    b->req[r].status = (unsigned *)base + q;
    if (grouped) {
      b->req[r].tscale = 1.0;
      if (gfix) set_fix_bits_raw(&b->req[r], grad, S->t_last32 - S->t_first32);
      launch_tiers(S->nrt, mode, true, &b->req[r].wide, &b->req[r].coarse);
    }
  }
  if (grouped) b->group = group_size(grad != 0, k);
  char *rows_cur = rows_base;
  if (direct_rows) {
    b->req[0].mu_out = mu_out;
    b->req[0].xi_out = xi_out;
  } else if (mu_out || xi_out) {
    b->req[0].mu_out = (double *)rows_cur;
    b->req[0].xi_out = (double *)(rows_cur + row_bytes);
    rows_cur += 2 * row_bytes;
  }
  char *pi_rows = pi_dev ? pi_dev : rows_cur;  // row q holds pi for params[q]
  if (pi_out || pi_dev)
    for (int r = 0; r < k; ++r) b->req[r].pi_out = (double *)(pi_rows + (size_t)order[r] * row_bytes);
  HK_CUDA(ctx, cudaMemsetAsync(base, 0, kFixedBytes + cnt, ctx->stream));
  if (int rc = launch_batch(ctx, *b, mode, grad, ctx->stream)) return rc;
  if (device_out) return HAWKES_OK;
  HK_CUDA(ctx, cudaMemcpyAsync(ctx->pinned_out, base, kHdrBytes + (size_t)k * kOut * sizeof(double),
                               cudaMemcpyDeviceToHost, ctx->stream));
  const size_t nb = (size_t)S->n * sizeof(double);
  std::vector<double *> dst;
  std::vector<const char *> src;
  if (mu_out && !direct_rows) { dst.push_back(mu_out); src.push_back((const char *)b->req[0].mu_out); }
  if (xi_out && !direct_rows) { dst.push_back(xi_out); src.push_back((const char *)b->req[0].xi_out); }
  if (pi_out)
    for (int q = 0; q < k; ++q) {
      dst.push_back(pi_out + (size_t)q * S->n);
      src.push_back(pi_rows + (size_t)q * row_bytes);
    }
  if (!dst.empty())
    if (int rc = rows_to_host(ctx, dst.data(), src.data(), (int)dst.size(), nb, ctx->stream)) return rc;
  HK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int q = 0; q < k; ++q)
    if (int rc = device_status(ctx->pinned_out, q)) return rc;
  std::memcpy(host_out, (const char *)ctx->pinned_out + kHdrBytes, (size_t)k * kOut * sizeof(double));
  return HAWKES_OK;
}

// ---- serving -------------------------------------------------------------------------

void complete_ticket(hawkes_ctx *ctx, uint64_t id, int status, const double *vals) {
  auto it = ctx->tickets.find(id);
  if (it == ctx->tickets.end()) return;
  TicketRec &T = it->second;
  T.status = status;
  T.done = true;
  T.t_done = now_ns();
  if (status == HAWKES_OK && vals) {
    T.ll = vals[0];
    for (int q = 0; q < 6; ++q) T.g[q] = vals[1 + q];
  }
  if (status == HAWKES_OK) ctx->n_completed++;
  else ctx->n_failed++;
}

void release_set_ref(hawkes_ctx *ctx, EventSetRec *S) {
  // caller holds ctx->mu
  if (--S->refs == 0 && S->released) {
    ctx->sets.erase(S->id);
    free_set(ctx, S);
  }
}

// Collect finished flights. Holds smu; takes mu briefly for set references.
void reap_flights(hawkes_ctx *ctx) {
  for (auto &F : ctx->flights) {
    if (!F.busy) continue;
    cudaError_t q = cudaEventQuery(F.done);
    if (q == cudaErrorNotReady) continue;
    const int status = q == cudaSuccess ? HAWKES_OK : HAWKES_E_CUDA;
    if (q != cudaSuccess) ctx->last_cuda = cudaGetErrorString(q);
    const double *vals = (const double *)((const char *)F.host_out + kHdrBytes);
    for (size_t r = 0; r < F.ids.size(); ++r) {
      const int st = status == HAWKES_OK ? device_status(F.host_out, (int)r) : status;
      complete_ticket(ctx, F.ids[r], st, vals + kOut * r);
    }
    {
      std::lock_guard<std::mutex> lock(ctx->mu);
      for (auto *S : F.sets) release_set_ref(ctx, S);
    }
    ctx->used -= F.ws_bytes;
    ctx->serving_bytes -= F.ws_bytes;
    F.ws = nullptr;
    F.ws_bytes = 0;
    F.ids.clear();
    F.sets.clear();
    F.busy = false;
    ctx->done_cv.notify_all();
  }
}

// Form and launch one batch on flight F from the pending queue. Holds smu.
// Returns true if a batch was launched.
bool launch_pending(hawkes_ctx *ctx, Flight &F) {
  if (ctx->pending.empty()) return false;
  const TicketRec &H = ctx->tickets[ctx->pending.front()];
  const int mode = H.mode, grad = H.grad;
  std::vector<uint64_t> take;
  std::vector<EventSetRec *> sets;
  size_t bytes = kFixedBytes, cnt = 0;
  const size_t used = ctx->used.load();
  const size_t room = ctx->budget > used ? ctx->budget - used : 0;
  const size_t fixed_used = used - ctx->serving_bytes;  // resident sets and the sync workspace
  bool any_flight = false;
  for (auto &G : ctx->flights) any_flight |= G.busy;
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    for (auto it = ctx->pending.begin(); it != ctx->pending.end() && (int)take.size() < kMaxBatch;) {
      TicketRec &T = ctx->tickets[*it];
      if (T.mode != mode || T.grad != grad) { ++it; continue; }
      auto sit = ctx->sets.find(T.set_id);
      if (sit == ctx->sets.end()) {  // cannot happen while the request holds a reference
        complete_ticket(ctx, *it, HAWKES_E_NOSET, nullptr);
        it = ctx->pending.erase(it);
        ctx->done_cv.notify_all();
        continue;
      }
      if (bytes + T.footprint + counter_bytes(sit->second, mode, grad, use_symmetry(sit->second, mode, T.flags)) > room) {
        const bool never_fits = kFixedBytes + 512 + T.footprint + counter_bytes(sit->second, mode, grad, use_symmetry(sit->second, mode, T.flags)) + fixed_used >
                                ctx->budget;
        if (take.empty() && !any_flight && never_fits) {
          complete_ticket(ctx, *it, HAWKES_E_ADMISSION, nullptr);
          release_set_ref(ctx, sit->second);
          it = ctx->pending.erase(it);
          ctx->done_cv.notify_all();
          continue;
        }
        break;  // first-come first-served within a kind: wait for memory to free up
      }
      bytes += T.footprint + counter_bytes(sit->second, mode, grad, use_symmetry(sit->second, mode, T.flags));
      cnt += counter_bytes(sit->second, mode, grad, use_symmetry(sit->second, mode, T.flags));
      take.push_back(*it);
      sets.push_back(sit->second);
      it = ctx->pending.erase(it);
    }
  }
  if (take.empty()) return false;
  const int64_t t_launch = now_ns();
  for (uint64_t id : take) ctx->tickets[id].t_launch = t_launch;
  void *ws = nullptr;
  std::unique_ptr<Batch> b(new Batch());
  std::memset(b.get(), 0, sizeof(Batch));
  int rc = HAWKES_OK;
  cnt = align_up(cnt, 256);
  bytes = align_up(bytes, 256) + 256;
  cudaError_t e = cudaMallocFromPoolAsync(&ws, bytes, ctx->pool, F.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws, 0, kFixedBytes + cnt, F.stream);
  if (e != cudaSuccess) rc = cuda_fail(ctx, e);
  if (rc == HAWKES_OK) {
    char *base = (char *)ws;
    double *outs = (double *)(base + kHdrBytes);
    char *cnt_cur = base + kFixedBytes;
    char *cur = base + kFixedBytes + cnt;
    b->nreq = (int)take.size();
    for (size_t r = 0; r < take.size() && rc == HAWKES_OK; ++r) {
      TicketRec &T = ctx->tickets[take[r]];
      rc = make_request(ctx, sets[r], &T.p, mode, grad, T.flags, &b->req[r]);
      bind_workspace(&b->req[r], sets[r], mode, grad, cur, outs + kOut * r, (unsigned *)cnt_cur, 1, b->req[r].sym);
      b->req[r].status = (unsigned *)base + r;
      cnt_cur += counter_bytes(sets[r], mode, grad, b->req[r].sym);
      cur += T.footprint;
    }
    if (rc == HAWKES_OK) rc = launch_batch(ctx, *b, mode, grad, F.stream);
    if (rc == HAWKES_OK) {
      e = cudaMemcpyAsync(F.host_out, base, kHdrBytes + take.size() * kOut * sizeof(double), cudaMemcpyDeviceToHost,
                          F.stream);
      if (e != cudaSuccess) rc = cuda_fail(ctx, e);
    }
    cudaFreeAsync(ws, F.stream);
    if (rc == HAWKES_OK) {
      e = cudaEventRecord(F.done, F.stream);
      if (e != cudaSuccess) rc = cuda_fail(ctx, e);
    }
  }
  if (rc != HAWKES_OK) {
    std::lock_guard<std::mutex> lock(ctx->mu);
    for (size_t r = 0; r < take.size(); ++r) {
      complete_ticket(ctx, take[r], rc, nullptr);
      release_set_ref(ctx, sets[r]);
    }
    ctx->done_cv.notify_all();
    return false;
  }
  ctx->used += bytes;
  ctx->serving_bytes += bytes;
  F.ws = ws;
  F.ws_bytes = bytes;
  F.ids = std::move(take);
  F.sets = std::move(sets);
  F.busy = true;
  ctx->n_launches++;
  return true;
}

void scheduler_loop(hawkes_ctx *ctx) {
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(ctx->smu);
  while (true) {
    reap_flights(ctx);
    bool launched = false;
    for (auto &F : ctx->flights) {
      if (F.busy || ctx->pending.empty()) continue;
      if (launch_pending(ctx, F)) launched = true;
    }
    bool inflight = false;
    for (auto &F : ctx->flights) inflight |= F.busy;
    if (ctx->shutdown && !inflight) break;
    if (launched) continue;
    if (inflight) ctx->scv.wait_for(lk, std::chrono::microseconds(20));
    else ctx->scv.wait_for(lk, std::chrono::milliseconds(50));
  }
}

int init_flights(hawkes_ctx *ctx) {
  if (ctx->flights_ready) return HAWKES_OK;
  for (auto &F : ctx->flights) {  // resumable: members created by an earlier failed call are kept
    if (!F.stream) HK_CUDA(ctx, cudaStreamCreateWithFlags(&F.stream, cudaStreamNonBlocking));
    if (!F.done) HK_CUDA(ctx, cudaEventCreateWithFlags(&F.done, cudaEventDisableTiming));
    if (!F.host_out) HK_CUDA(ctx, cudaMallocHost((void **)&F.host_out, kFixedBytes));
  }
  ctx->flights_ready = true;
  return HAWKES_OK;
}

}  // namespace

// ---- public ABI ------------------------------------------------------------------------

extern "C" {

const char *hawkes_strerror(int status) {
  switch (status) {
    case HAWKES_OK: return "ok";
    case HAWKES_E_INVAL: return "invalid argument";
    case HAWKES_E_UNSORTED: return "event times are not sorted";
    case HAWKES_E_NOSET: return "unknown event set";
    case HAWKES_E_ADMISSION: return "device memory budget exceeded";
    case HAWKES_E_NOMEM: return "out of memory";
    case HAWKES_E_TIMEOUT: return "timed out";
    case HAWKES_E_PENDING: return "pending";
    case HAWKES_E_CUDA: return "CUDA error";
    case HAWKES_E_TICKET: return "unknown or consumed ticket";
    case HAWKES_E_SHUTDOWN: return "context shut down";
    case HAWKES_E_DEVICE: return "a bounded device wait ran out (results discarded)";
    default: return "unknown status";
  }
}

const char *hawkes_last_cuda_error(hawkes_ctx *ctx) { return ctx ? ctx->last_cuda.c_str() : ""; }

int hawkes_create(hawkes_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream) {
  if (!out) return HAWKES_E_INVAL;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e);
  if (device < 0 || device >= ndev) return HAWKES_E_INVAL;
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(nullptr, e);
  std::unique_ptr<hawkes_ctx> ctx(new (std::nothrow) hawkes_ctx());
  if (!ctx) return HAWKES_E_NOMEM;
  ctx->device = device;
  e = init_log_table();
  if (e != cudaSuccess) return cuda_fail(nullptr, e);
  cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaDeviceGetAttribute(&ctx->host_direct, cudaDevAttrPageableMemoryAccess, device) != cudaSuccess)
    ctx->host_direct = 0;
  ctx->occ_launch[1][0] = occupancy_pair_mixed(false);
  ctx->occ_launch[1][1] = occupancy_pair_mixed(true);
  ctx->occ_launch[0][0] = occupancy_pair_fp64(false);
  ctx->occ_launch[0][1] = occupancy_pair_fp64(true);
  ctx->occ[0] = ctx->occ_launch[1][0];
  ctx->occ[1] = ctx->occ_launch[1][1];
  ctx->occ[2] = std::min(ctx->occ_launch[0][0], ctx->occ_launch[0][1]);
  for (int &o : ctx->occ) o = std::max(1, o);
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(nullptr, e);
    ctx->own_stream = true;
  }
  size_t free_b = 0, total_b = 0;
  e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) return cuda_fail(nullptr, e);
  ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)free_b);
  e = cudaMallocHost((void **)&ctx->pinned_out, kFixedBytes);
  if (e != cudaSuccess) return cuda_fail(nullptr, e);
  // the context's own device memory pool; it keeps freed memory for reuse (the HBM budget
  // bounds what the context holds) and returns it when the context is destroyed
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  e = cudaMemPoolCreate(&ctx->pool, &props);
  if (e != cudaSuccess) {
    cudaFreeHost(ctx->pinned_out);
    return cuda_fail(nullptr, e);
  }
  uint64_t keep = ~(uint64_t)0;
  cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  *out = ctx.release();
  return HAWKES_OK;
}

int hawkes_destroy(hawkes_ctx *ctx) {
  if (!ctx) return HAWKES_OK;
  cudaSetDevice(ctx->device);
  {
    std::unique_lock<std::mutex> lk(ctx->smu);
    ctx->shutdown = true;
    for (uint64_t id : ctx->pending) complete_ticket(ctx, id, HAWKES_E_SHUTDOWN, nullptr);
    {
      std::lock_guard<std::mutex> lock(ctx->mu);
      for (uint64_t id : ctx->pending) {
        auto it = ctx->sets.find(ctx->tickets[id].set_id);
        if (it != ctx->sets.end()) it->second->refs--;
      }
    }
    ctx->pending.clear();
    ctx->scv.notify_all();
    ctx->done_cv.notify_all();
  }
  if (ctx->sched_thread.joinable()) ctx->sched_thread.join();
  cudaStreamSynchronize(ctx->stream);
  for (auto &F : ctx->flights) {
    if (F.stream) { cudaStreamSynchronize(F.stream); cudaStreamDestroy(F.stream); }
    if (F.done) cudaEventDestroy(F.done);
    if (F.host_out) cudaFreeHost(F.host_out);
  }
  for (cudaEvent_t ev : ctx->kev)
    if (ev) cudaEventDestroy(ev);
  for (auto &kv : ctx->sets) {
    if (kv.second->dev) cudaFreeAsync(kv.second->dev, ctx->stream);
    delete kv.second;
  }
  ctx->sets.clear();
  cudaStreamSynchronize(ctx->stream);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  if (ctx->sync_ws.dev) cudaFree(ctx->sync_ws.dev);
  if (ctx->pinned_out) cudaFreeHost(ctx->pinned_out);
  if (ctx->stage) cudaFreeHost(ctx->stage);
  if (ctx->bounce) cudaFreeHost(ctx->bounce);
  for (cudaEvent_t ev : ctx->bounce_ev)
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : ctx->chunk_ev) cudaEventDestroy(ev);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return HAWKES_OK;
}

int hawkes_set_flags(hawkes_ctx *ctx, int flags) {
  if (!ctx || (flags & ~(HAWKES_FLAG_EXCLUDE_SELF | HAWKES_FLAG_DENSE | HAWKES_FLAG_NO_SYMMETRY |
                         HAWKES_FLAG_TEST_WITHHOLD_READY)))
    return HAWKES_E_INVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  ctx->flags = flags;
  return HAWKES_OK;
}

int hawkes_upload_events(hawkes_ctx *ctx, const double *x, const double *y, const double *t, int64_t n,
                         int32_t *set_id_out) {
  if (!ctx || !x || !y || !t || !set_id_out || n < 1) return HAWKES_E_INVAL;
  if (n > (int64_t)1 << 30) return HAWKES_E_INVAL;
  cudaSetDevice(ctx->device);
  const int64_t npad = (int64_t)align_up((size_t)n, kPadTo);
  std::unique_ptr<EventSetRec> S(new EventSetRec());
  S->n = n;
  S->npad = npad;
  S->nrt = (int)(npad / kRowTile);
  S->nct = (int)(npad / kColTile);
  for (int k = 0; k < kKinds; ++k) {
    // the float64 kernel can cut a column tile into chunks, the mixed kernels cannot
    const int units = k == kind_of(HAWKES_FP64, 0) ? S->nct * fp64_chunks_per_tile() : S->nct;
    S->slices[k] = slices_for(S->nrt, units, ctx->sms * ctx->occ[k], k != kind_of(HAWKES_FP64, 0));
  }
  // One device allocation. The caller's float64 coordinates are copied in, and one launch
  // (launch_upload_prep) forms the rest and checks the inputs into a flag word.
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes, 256); return o; };
  const size_t o_x64 = take(npad * 8), o_y64 = take(npad * 8), o_t64 = take(npad * 8), o_flag = take(4);
  const size_t o_x32 = take(npad * 4), o_y32 = take(npad * 4), o_t32 = take(npad * 4);
  const size_t o_lo32 = take(npad * 4), o_lo64 = take(npad * 4);
  const size_t o_w32 = take((size_t)2 * kWinBuckets * 4), o_w64 = take((size_t)2 * kWinBuckets * 4);
  const size_t bytes = off;
  // window tables: none when the times span too little for buckets wider than their rounding
  auto table = [&](double t0, double t1, WinTable *W, double *width) {
    *W = WinTable{};
    const double span = t1 - t0, scale = std::max({std::fabs(t0), std::fabs(t1), 1.0});
    if (!(span > 1e-9 * scale)) return false;
    *width = span / kWinBuckets;
    W->t0 = t0;
    W->inv = 1.0 / *width;
    W->nb = kWinBuckets;
    return true;
  };
  UploadPrep u{};
  S->t_first64 = t[0]; S->t_last64 = t[n - 1];
  S->t_first32 = (double)(float)t[0]; S->t_last32 = (double)(float)t[n - 1];
  const bool tab32 = table(S->t_first32, S->t_last32, &S->win32, &u.width_32);
  const bool tab64 = table(S->t_first64, S->t_last64, &S->win64, &u.width_64);
  u.t0_32 = S->t_first32;
  u.t0_64 = S->t_first64;
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (ctx->used.load() + bytes > ctx->budget) return HAWKES_E_ADMISSION;
  if (!ctx->stage) {  // pinned word for the check flags, kept for later uploads
    cudaError_t es = cudaMallocHost((void **)&ctx->stage, 256);
    if (es != cudaSuccess) {
      ctx->stage = nullptr;
      return cuda_fail(ctx, es);
    }
  }
  unsigned *hflag = (unsigned *)ctx->stage;
  *hflag = 0u;
  void *dev = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&dev, bytes, ctx->pool, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e);
  char *d = (char *)dev;
  u.x64 = (double *)(d + o_x64); u.y64 = (double *)(d + o_y64); u.t64 = (double *)(d + o_t64);
  u.x32 = (float *)(d + o_x32); u.y32 = (float *)(d + o_y32); u.t32 = (float *)(d + o_t32);
  u.lo32 = (int *)(d + o_lo32); u.lo64 = (int *)(d + o_lo64);
  u.w32 = tab32 ? (int *)(d + o_w32) : nullptr;
  u.w64 = tab64 ? (int *)(d + o_w64) : nullptr;
  u.flags = (unsigned *)(d + o_flag);
  u.n = n;
  u.npad = npad;
  u.sms = ctx->sms;
  if (ctx->host_direct) {  // the launch reads the caller's arrays in place (coherent host memory)
    u.sx = x; u.sy = y; u.st = t;
  } else {  // copied straight from the caller's (pageable) arrays, then read on the device
    u.sx = u.x64; u.sy = u.y64; u.st = u.t64;
    e = cudaMemcpyAsync(u.x64, x, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u.y64, y, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u.t64, t, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(u.flags, 0, sizeof(unsigned), ctx->stream);
  if (e == cudaSuccess) e = launch_upload_prep(u, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hflag, u.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(dev, ctx->stream);
    return cuda_fail(ctx, e);
  }
  if (*hflag) {  // checks of Section 2.1's domain: finite coordinates, times in [0, inf), sorted
    cudaFreeAsync(dev, ctx->stream);
    return (*hflag & 1u) ? HAWKES_E_INVAL : HAWKES_E_UNSORTED;
  }
  S->dev = dev;
  S->bytes = bytes;
  S->x32 = (float *)(d + o_x32); S->y32 = (float *)(d + o_y32); S->t32 = (float *)(d + o_t32);
  S->x64 = (double *)(d + o_x64); S->y64 = (double *)(d + o_y64); S->t64 = (double *)(d + o_t64);
  S->lo32 = (int *)(d + o_lo32); S->lo64 = (int *)(d + o_lo64);
  if (S->win32.nb) { S->win32.first = (int *)(d + o_w32); S->win32.last = S->win32.first + S->win32.nb; }
  if (S->win64.nb) { S->win64.first = (int *)(d + o_w64); S->win64.last = S->win64.first + S->win64.nb; }
  ctx->used += bytes;
  const int32_t id = ctx->next_set++;
  S->id = id;
  ctx->sets[id] = S.release();
  *set_id_out = id;
  return HAWKES_OK;
}

int hawkes_release_events(hawkes_ctx *ctx, int32_t set_id) {
  if (!ctx) return HAWKES_E_INVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  auto it = ctx->sets.find(set_id);
  if (it == ctx->sets.end() || it->second->released) return HAWKES_E_NOSET;
  EventSetRec *S = it->second;
  S->released = true;
  if (S->refs == 0) {
    cudaStreamSynchronize(ctx->stream);
    ctx->sets.erase(it);
    free_set(ctx, S);
  }
  return HAWKES_OK;
}

int hawkes_set_info(hawkes_ctx *ctx, int32_t set_id, int64_t *n_out, size_t *device_bytes_out) {
  if (!ctx) return HAWKES_E_INVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  EventSetRec *S = find_set(ctx, set_id);
  if (!S) return HAWKES_E_NOSET;
  if (n_out) *n_out = S->n;
  if (device_bytes_out) *device_bytes_out = S->bytes;
  return HAWKES_OK;
}

int hawkes_pair_work(hawkes_ctx *ctx, int32_t set_id, const hawkes_params *params, hawkes_mode mode,
                     int64_t out[5]) {
  if (!ctx || !params || !out || (mode != HAWKES_FP64 && mode != HAWKES_MIXED)) return HAWKES_E_INVAL;
  if (int rc = check_params(params)) return rc;
  std::lock_guard<std::mutex> lock(ctx->mu);
  EventSetRec *S = find_set(ctx, set_id);
  if (!S) return HAWKES_E_NOSET;
  Request R;
  if (int rc = make_request(ctx, S, params, mode, 0, ctx->flags, &R)) return rc;
  const int64_t n = S->n;
  // stored times of the mode, as doubles
  std::vector<double> t((size_t)n);
  if (mode == HAWKES_MIXED) {
    std::vector<float> t32((size_t)n);
    HK_CUDA(ctx, cudaMemcpyAsync(t32.data(), S->t32, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    HK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int64_t i = 0; i < n; ++i) t[(size_t)i] = (double)t32[(size_t)i];
  } else {
    HK_CUDA(ctx, cudaMemcpyAsync(t.data(), S->t64, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    HK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  // reach (days) of each term on its own (the window uses the larger on the early side)
  double bg_reach, trig_reach;
  term_reaches(params, mode, R.beta, ctx->flags, n, &bg_reach, &trig_reach);
  int64_t visited = 0, bg_pairs = 0, trig_pairs = 0;
  WinTable W = mode == HAWKES_MIXED ? S->win32 : S->win64;  // the kernels' table, read back
  std::vector<int> wh((size_t)2 * W.nb);
  if (W.nb) {
    HK_CUDA(ctx, cudaMemcpyAsync(wh.data(), W.first, wh.size() * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    W.first = wh.data();
    W.last = wh.data() + W.nb;
  }
  int64_t evaluated = 0;
  auto cols_in = [&](int c0, int c1) {  // real columns of column tiles [c0, c1)
    return std::max<int64_t>(0, std::min<int64_t>((int64_t)c1 * kColTile, n) - (int64_t)c0 * kColTile);
  };
  for (int rt = 0; rt < S->nrt; ++rt) {  // the window the kernels use (table_window_rt)
    const int64_t r0 = (int64_t)rt * kRowTile, r1 = std::min<int64_t>(r0 + kRowTile, n) - 1;
    int c0 = 0, c1 = S->nct;
    if (!(ctx->flags & HAWKES_FLAG_DENSE) && W.nb) {
      const int2 w = table_window(W, (int)n, S->nct, t[(size_t)r0] - R.cut_early, t[(size_t)r1] + R.cut_late);
      c0 = w.x;
      c1 = w.y;
    } else if (!(ctx->flags & HAWKES_FLAG_DENSE)) {
      const int64_t j0 = std::lower_bound(t.begin(), t.end(), t[(size_t)r0] - R.cut_early) - t.begin();
      const int64_t j1 = std::upper_bound(t.begin(), t.end(), t[(size_t)r1] + R.cut_late) - t.begin();
      c0 = (int)(j0 / kColTile);
      c1 = std::max(std::min((int)((j1 + kColTile - 1) / kColTile), S->nct), c0 + 1);
    }
    if (R.sym) {  // far (and shared near) column tiles serve both events of a pair (SymPlan)
      const SymPlan pl = sym_plan_scan(R, W, rt, make_int2(c0, c1), [&](int K) { return t[(size_t)K * kRowTile]; });
      visited += (r1 - r0 + 1) * (cols_in(c0, pl.end) + cols_in(c0, pl.near_end));
      evaluated += (r1 - r0 + 1) * cols_in(c0, pl.end);
    } else {
      visited += (r1 - r0 + 1) * cols_in(c0, c1);
      evaluated += (r1 - r0 + 1) * cols_in(c0, c1);
    }
  }
  for (int64_t i = 0; i < n; ++i) {  // pairs whose term can be nonzero at the working precision
    const double ti = t[(size_t)i];
    bg_pairs += (std::upper_bound(t.begin(), t.end(), ti + bg_reach) - t.begin()) -
                (std::lower_bound(t.begin(), t.end(), ti - bg_reach) - t.begin());
    trig_pairs += (std::lower_bound(t.begin(), t.end(), ti) - t.begin()) -
                  (std::lower_bound(t.begin(), t.end(), ti - trig_reach) - t.begin());
  }
  out[0] = visited;
  out[1] = n * n;
  out[2] = bg_pairs;
  out[3] = trig_pairs;
  out[4] = evaluated;
  return HAWKES_OK;
}

int hawkes_loglik(hawkes_ctx *ctx, int32_t set_id, const hawkes_params *params, hawkes_mode mode,
                  double *loglik_out) {
  if (!ctx || !params || !loglik_out) return HAWKES_E_INVAL;
  cudaSetDevice(ctx->device);
  double out[kOut];
  int rc = eval_sync(ctx, set_id, 1, params, mode, 0, out, nullptr, nullptr, nullptr, nullptr);
  if (rc == HAWKES_OK) *loglik_out = out[0];
  return rc;
}

int hawkes_loglik_grad(hawkes_ctx *ctx, int32_t set_id, const hawkes_params *params, hawkes_mode mode,
                       double *loglik_out, double grad_out[6]) {
  if (!ctx || !params || !loglik_out || !grad_out) return HAWKES_E_INVAL;
  cudaSetDevice(ctx->device);
  double out[kOut];
  int rc = eval_sync(ctx, set_id, 1, params, mode, 1, out, nullptr, nullptr, nullptr, nullptr);
  if (rc == HAWKES_OK) {
    *loglik_out = out[0];
    for (int q = 0; q < 6; ++q) grad_out[q] = out[1 + q];
  }
  return rc;
}

int hawkes_loglik_mix(hawkes_ctx *ctx, int32_t set_id, const hawkes_mix_params *params, int m, hawkes_mode mode,
                      int want_grad, double *loglik_out, double *grad_out) {
  if (!ctx || !params || !loglik_out || (want_grad && !grad_out) || m < 1 || m > HAWKES_MIX_MAX)
    return HAWKES_E_INVAL;
  cudaSetDevice(ctx->device);
  const hawkes_params p1{params->mu0, params->tau_x, params->tau_t, params->theta[0], params->omega[0], params->h[0]};
  double out[kOut];
  const int rc = eval_sync(ctx, set_id, 1, &p1, mode, want_grad ? 1 : 0, out, nullptr, nullptr, nullptr, nullptr,
                           m > 1 ? params : nullptr);
  if (rc != HAWKES_OK) return rc;
  *loglik_out = out[0];
  if (want_grad)
    for (int q = 0; q < 3 + 3 * m; ++q) grad_out[q] = out[1 + q];
  return HAWKES_OK;
}

int hawkes_loglik_async(hawkes_ctx *ctx, int32_t set_id, const hawkes_params *params, hawkes_mode mode,
                        int want_grad, double *device_out) {
  if (!ctx || !params || !device_out) return HAWKES_E_INVAL;
  cudaSetDevice(ctx->device);
  return eval_sync(ctx, set_id, 1, params, mode, want_grad ? 1 : 0, nullptr, device_out, nullptr, nullptr, nullptr);
}

int hawkes_loglik_batch(hawkes_ctx *ctx, int32_t set_id, int k, const hawkes_params *params, hawkes_mode mode,
                        int want_grad, double *loglik_out, double *grad_out) {
  if (!ctx || !params || !loglik_out || (want_grad && !grad_out) || k < 1 || k > kMaxBatch)
    return HAWKES_E_INVAL;
  cudaSetDevice(ctx->device);
  std::vector<double> out((size_t)k * kOut);
  int rc = eval_sync(ctx, set_id, k, params, mode, want_grad ? 1 : 0, out.data(), nullptr, nullptr, nullptr, nullptr);
  if (rc != HAWKES_OK) return rc;
  for (int r = 0; r < k; ++r) {
    loglik_out[r] = out[(size_t)r * kOut];
    if (want_grad)
      for (int q = 0; q < 6; ++q) grad_out[(size_t)r * 6 + q] = out[(size_t)r * kOut + 1 + q];
  }
  return HAWKES_OK;
}

int hawkes_event_terms(hawkes_ctx *ctx, int32_t set_id, const hawkes_params *params, hawkes_mode mode,
                       double *mu_out, double *xi_out, double *loglik_out) {
  if (!ctx || !params || !mu_out || !xi_out) return HAWKES_E_INVAL;
  cudaSetDevice(ctx->device);
  double out[kOut];
  int rc = eval_sync(ctx, set_id, 1, params, mode, 0, out, nullptr, mu_out, xi_out, nullptr);
  if (rc == HAWKES_OK && loglik_out) *loglik_out = out[0];
  return rc;
}

int hawkes_pi_batch(hawkes_ctx *ctx, int32_t set_id, int k, const hawkes_params *params, hawkes_mode mode,
                    double *pi_out, double *loglik_out) {
  if (!ctx || !params || !pi_out || k < 0) return HAWKES_E_INVAL;
  if (mode != HAWKES_FP64 && mode != HAWKES_MIXED) return HAWKES_E_INVAL;
  for (int r = 0; r < k; ++r)
    if (int rc = check_params(&params[r])) return rc;
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> lock(ctx->mu);
  EventSetRec *S = find_set(ctx, set_id);
  if (!S) return HAWKES_E_NOSET;
  if (k == 0) return HAWKES_OK;
  // Every launch of up to kMaxBatch parameter vectors is enqueued first, with its pi rows in
  // one device buffer; the rows of launch c leave through the bounce buffer on a second
  // stream as soon as launch c is done, while the later launches run.
  const size_t row_bytes = align_up((size_t)S->n * sizeof(double), 256);
  const size_t outs_off = align_up((size_t)k * row_bytes, 256);
  const int chunks = (k + kMaxBatch - 1) / kMaxBatch;
  if (!ctx->copy_stream) HK_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  while ((int)ctx->chunk_ev.size() < chunks) {
    cudaEvent_t ev = nullptr;
    HK_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    ctx->chunk_ev.push_back(ev);
  }
  if (ctx->used.load() + outs_off + (size_t)k * kOut * sizeof(double) > ctx->budget) return HAWKES_E_ADMISSION;
  const size_t dev_bytes = outs_off + (size_t)k * kOut * sizeof(double);
  void *dev = nullptr;
  HK_CUDA(ctx, cudaMallocFromPoolAsync(&dev, dev_bytes, ctx->pool, ctx->stream));
  ctx->used += dev_bytes;
  char *rows = (char *)dev;
  double *outs = (double *)(rows + outs_off);
  int rc = HAWKES_OK;
  int launched = 0;
  for (int c = 0; c < chunks && rc == HAWKES_OK; ++c, ++launched) {
    const int r0 = c * kMaxBatch, m = std::min(kMaxBatch, k - r0);
    rc = eval_locked(ctx, S, m, params + r0, mode, 0, nullptr, outs + (size_t)kOut * r0, nullptr, nullptr, nullptr,
                     rows + (size_t)r0 * row_bytes);
    if (rc == HAWKES_OK && cudaEventRecord(ctx->chunk_ev[c], ctx->stream) != cudaSuccess) rc = HAWKES_E_CUDA;
  }
  std::vector<double *> dst;
  std::vector<const char *> src;
  for (int c = 0; c < launched && rc == HAWKES_OK; ++c) {
    const int r0 = c * kMaxBatch, m = std::min(kMaxBatch, k - r0);
    if (cudaStreamWaitEvent(ctx->copy_stream, ctx->chunk_ev[c], 0) != cudaSuccess) { rc = HAWKES_E_CUDA; break; }
    dst.clear();
    src.clear();
    for (int r = r0; r < r0 + m; ++r) {
      dst.push_back(pi_out + (size_t)r * S->n);
      src.push_back(rows + (size_t)r * row_bytes);
    }
    rc = rows_to_host(ctx, dst.data(), src.data(), m, (size_t)S->n * sizeof(double), ctx->copy_stream);
  }
  std::vector<double> host((size_t)k * kOut);
  if (rc == HAWKES_OK && cudaMemcpyAsync(host.data(), outs, host.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                         ctx->stream) != cudaSuccess)
    rc = HAWKES_E_CUDA;
  const cudaError_t e1 = cudaStreamSynchronize(ctx->copy_stream), e2 = cudaStreamSynchronize(ctx->stream);
  cudaFreeAsync(dev, ctx->stream);
  ctx->used -= dev_bytes;
  if (rc != HAWKES_OK) return rc;
  if (e1 != cudaSuccess) return cuda_fail(ctx, e1);
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2);
  for (int r = 0; r < k; ++r)  // the status words of earlier launches are cleared by later ones:
    if (std::isnan(host[(size_t)kOut * r])) return HAWKES_E_DEVICE;  // a NaN ell is a device wait that ran out
  if (loglik_out)
    for (int r = 0; r < k; ++r) loglik_out[r] = host[(size_t)kOut * r];
  return HAWKES_OK;
}

int hawkes_submit(hawkes_ctx *ctx, int32_t set_id, const hawkes_params *params, int want_grad, hawkes_mode mode,
                  uint64_t *ticket_out) {
  if (!ctx || !params || !ticket_out) return HAWKES_E_INVAL;
  if (mode != HAWKES_FP64 && mode != HAWKES_MIXED) return HAWKES_E_INVAL;
  if (int rc = check_params(params)) return rc;
  cudaSetDevice(ctx->device);
  TicketRec T;
  T.set_id = set_id;
  T.p = *params;
  T.grad = want_grad ? 1 : 0;
  T.mode = mode;
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    EventSetRec *S = find_set(ctx, set_id);
    if (!S) return HAWKES_E_NOSET;
    Request probe;
    if (int rc = make_request(ctx, S, params, mode, T.grad, ctx->flags, &probe)) return rc;
    T.flags = ctx->flags;
    T.footprint = request_footprint(S, mode, T.grad, 1, probe.sym);
    if (T.footprint + counter_bytes(S, mode, T.grad, probe.sym) + 4096 > ctx->budget) return HAWKES_E_ADMISSION;
    S->refs++;
  }
  std::lock_guard<std::mutex> lk(ctx->smu);
  if (ctx->shutdown) {
    std::lock_guard<std::mutex> lock(ctx->mu);
    auto it = ctx->sets.find(set_id);
    if (it != ctx->sets.end()) release_set_ref(ctx, it->second);
    return HAWKES_E_SHUTDOWN;
  }
  if (int rc = init_flights(ctx)) {
    std::lock_guard<std::mutex> lock(ctx->mu);
    auto it = ctx->sets.find(set_id);
    if (it != ctx->sets.end()) release_set_ref(ctx, it->second);
    return rc;
  }
  const uint64_t id = ctx->next_ticket++;
  T.t_submit = now_ns();
  ctx->tickets[id] = T;
  ctx->pending.push_back(id);
  ctx->n_submitted++;
  if (!ctx->sched_running) {
    ctx->sched_running = true;
    ctx->sched_thread = std::thread(scheduler_loop, ctx);
  }
  ctx->scv.notify_all();
  *ticket_out = id;
  return HAWKES_OK;
}

int hawkes_poll_timed(hawkes_ctx *ctx, uint64_t ticket, int *done_out, double *loglik_out, double grad_out[6],
                      int64_t *queued_ns_out, int64_t *total_ns_out) {
  if (!ctx || !done_out) return HAWKES_E_INVAL;
  std::lock_guard<std::mutex> lk(ctx->smu);
  auto it = ctx->tickets.find(ticket);
  if (it == ctx->tickets.end()) return HAWKES_E_TICKET;
  if (!it->second.done) {
    *done_out = 0;
    return HAWKES_E_PENDING;
  }
  *done_out = 1;
  const TicketRec T = it->second;
  ctx->tickets.erase(it);
  if (queued_ns_out) *queued_ns_out = (T.t_launch ? T.t_launch : T.t_done) - T.t_submit;
  if (total_ns_out) *total_ns_out = T.t_done - T.t_submit;
  if (T.status != HAWKES_OK) return T.status;
  if (loglik_out) *loglik_out = T.ll;
  if (grad_out)
    for (int q = 0; q < 6; ++q) grad_out[q] = T.grad ? T.g[q] : 0.0;
  return HAWKES_OK;
}

int hawkes_poll(hawkes_ctx *ctx, uint64_t ticket, int *done_out, double *loglik_out, double grad_out[6]) {
  if (!ctx || !done_out) return HAWKES_E_INVAL;
  std::lock_guard<std::mutex> lk(ctx->smu);
  auto it = ctx->tickets.find(ticket);
  if (it == ctx->tickets.end()) return HAWKES_E_TICKET;
  if (!it->second.done) {
    *done_out = 0;
    return HAWKES_E_PENDING;
  }
  *done_out = 1;
  const TicketRec T = it->second;
  ctx->tickets.erase(it);
  if (T.status != HAWKES_OK) return T.status;
  if (loglik_out) *loglik_out = T.ll;
  if (grad_out)
    for (int q = 0; q < 6; ++q) grad_out[q] = T.grad ? T.g[q] : 0.0;
  return HAWKES_OK;
}

int hawkes_wait(hawkes_ctx *ctx, uint64_t ticket, int timeout_ms, double *loglik_out, double grad_out[6]) {
  if (!ctx) return HAWKES_E_INVAL;
  std::unique_lock<std::mutex> lk(ctx->smu);
  auto ready = [&] {
    auto it = ctx->tickets.find(ticket);
    return it == ctx->tickets.end() || it->second.done;
  };
  if (timeout_ms < 0) ctx->done_cv.wait(lk, ready);
  else if (!ctx->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return HAWKES_E_TIMEOUT;
  auto it = ctx->tickets.find(ticket);
  if (it == ctx->tickets.end()) return HAWKES_E_TICKET;
  const TicketRec T = it->second;
  ctx->tickets.erase(it);
  if (T.status != HAWKES_OK) return T.status;
  if (loglik_out) *loglik_out = T.ll;
  if (grad_out)
    for (int q = 0; q < 6; ++q) grad_out[q] = T.grad ? T.g[q] : 0.0;
  return HAWKES_OK;
}

int hawkes_set_kernel_timing(hawkes_ctx *ctx, int on) {
  if (!ctx) return HAWKES_E_INVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  cudaSetDevice(ctx->device);
  if (on && !ctx->kev[0])
    for (cudaEvent_t &ev : ctx->kev) HK_CUDA(ctx, cudaEventCreate(&ev));
  ctx->ktime = on ? 1 : 0;
  ctx->kev_recorded = 0;
  return HAWKES_OK;
}

int hawkes_kernel_ms(hawkes_ctx *ctx, double ms_out[2]) {
  if (!ctx || !ms_out) return HAWKES_E_INVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (!ctx->kev_recorded) return HAWKES_E_PENDING;
  cudaSetDevice(ctx->device);
  HK_CUDA(ctx, cudaEventSynchronize(ctx->kev[2]));
  float a = 0.f, b = 0.f;
  HK_CUDA(ctx, cudaEventElapsedTime(&a, ctx->kev[0], ctx->kev[1]));
  HK_CUDA(ctx, cudaEventElapsedTime(&b, ctx->kev[1], ctx->kev[2]));
  ms_out[0] = a;
  ms_out[1] = b;
  return HAWKES_OK;
}

int hawkes_stats(hawkes_ctx *ctx, int64_t out[7]) {
  if (!ctx || !out) return HAWKES_E_INVAL;
  std::lock_guard<std::mutex> lk(ctx->smu);
  int64_t inflight = 0;
  for (auto &F : ctx->flights) inflight += F.busy ? (int64_t)F.ids.size() : 0;
  out[0] = ctx->n_submitted;
  out[1] = ctx->n_completed;
  out[2] = ctx->n_failed;
  out[3] = ctx->n_launches;
  out[4] = inflight;
  out[5] = (int64_t)ctx->pending.size();
  out[6] = (int64_t)ctx->serving_bytes;
  return HAWKES_OK;
}

}  // extern "C"
