// A fake CUDA runtime for testing the library's host logic on a machine without a GPU.
//
// Test infrastructure only. The library's host runtime (api.cu, compiled here as plain
// C++) is linked against this file instead of libcudart: "device" memory is host memory,
// streams and events are counters, and the kernel launchers are replaced by stubs that
// (1) check the work decomposition of every request (item counts, slices, window cut-offs,
// workspace pointers) and
// (2) write a recognisable value per request into its output so the tests can check that
// results reach the right ticket. No likelihood arithmetic happens here.
//
// Fault injection: fake_fail_alloc_after(k) makes the k-th following allocation fail;
// fake_event_delay(k) makes every event report "not ready" k times before completing;
// fake_release_events() completes every event recorded so far.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../paper_2005_10123_gb300/csrc/upload.h"

namespace {
std::atomic<long> g_fail_after{-1};
std::atomic<int> g_event_delay{0};
std::atomic<long> g_schedule_errors{0};
std::atomic<int> g_last_group{0};
std::atomic<long> g_group_launches{0};
std::atomic<long> g_sym_checked{0};  // launches whose shared-background plan was checked in full
std::atomic<long> g_launches{0};
std::atomic<long> g_live_allocs{0};
std::mutex g_mu;
std::atomic<long> g_epoch{0};  // events recorded before fake_release_events() complete
struct FakeEvent { int remaining; long epoch; };

bool alloc_fails() {
  long v = g_fail_after.load();
  if (v < 0) return false;
  if (v == 0) { g_fail_after = -1; return true; }
  g_fail_after = v - 1;
  return false;
}
}  // namespace

extern "C" {
void fake_fail_alloc_after(long k) { g_fail_after = k; }
void fake_event_delay(int k) { g_event_delay = k; }
void fake_release_events() { g_epoch++; }
long fake_schedule_errors() { return g_schedule_errors.load(); }
int fake_last_group() { return g_last_group.load(); }
long fake_group_launches() { return g_group_launches.load(); }
long fake_sym_checked() { return g_sym_checked.load(); }
long fake_launches() { return g_launches.load(); }
long fake_live_allocs() { return g_live_allocs.load(); }

cudaError_t cudaGetDeviceCount(int *c) { *c = 1; return cudaSuccess; }
cudaError_t cudaSetDevice(int) { return cudaSuccess; }
cudaError_t cudaDeviceGetAttribute(int *v, cudaDeviceAttr a, int) {
  *v = 0;
  if (a == cudaDevAttrMultiProcessorCount) *v = 152;
  // host memory is the fake's device memory: a device that reads pageable host memory, or
  // not, as the test asks (FAKE_HOST_DIRECT=1)
  if (a == cudaDevAttrPageableMemoryAccess) {
    const char *e = std::getenv("FAKE_HOST_DIRECT");
    *v = e && e[0] == '1';
  }
  return cudaSuccess;
}
cudaError_t cudaMemGetInfo(size_t *f, size_t *t) { *f = (size_t)64 << 30; *t = (size_t)80 << 30; return cudaSuccess; }
const char *cudaGetErrorString(cudaError_t e) { return e == cudaSuccess ? "no error" : "fake cuda error"; }
cudaError_t cudaMalloc(void **p, size_t n) {
  if (alloc_fails()) return cudaErrorMemoryAllocation;
  *p = std::aligned_alloc(256, (n + 255) / 256 * 256);
  if (!*p) return cudaErrorMemoryAllocation;
  std::memset(*p, 0xA5, n);  // garbage, as fresh device memory would be
  g_live_allocs++;
  return cudaSuccess;
}
cudaError_t cudaMallocAsync(void **p, size_t n, cudaStream_t) { return cudaMalloc(p, n); }
cudaError_t cudaMallocFromPoolAsync(void **p, size_t n, cudaMemPool_t, cudaStream_t) { return cudaMalloc(p, n); }
cudaError_t cudaMemPoolCreate(cudaMemPool_t *pool, const cudaMemPoolProps *) {
  static int token;
  *pool = reinterpret_cast<cudaMemPool_t>(&token);
  g_live_allocs++;
  return cudaSuccess;
}
cudaError_t cudaMemPoolDestroy(cudaMemPool_t) { g_live_allocs--; return cudaSuccess; }
cudaError_t cudaMemPoolSetAttribute(cudaMemPool_t, cudaMemPoolAttr, void *) { return cudaSuccess; }
cudaError_t cudaFree(void *p) { if (p) { std::free(p); g_live_allocs--; } return cudaSuccess; }
cudaError_t cudaFreeAsync(void *p, cudaStream_t) { return cudaFree(p); }
cudaError_t cudaMallocHost(void **p, size_t n) {
  if (alloc_fails()) return cudaErrorMemoryAllocation;
  *p = std::malloc(n);
  g_live_allocs++;
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaFreeHost(void *p) { if (p) { std::free(p); g_live_allocs--; } return cudaSuccess; }
cudaError_t cudaMemcpyAsync(void *d, const void *s, size_t n, cudaMemcpyKind, cudaStream_t) {
  std::memcpy(d, s, n);
  return cudaSuccess;
}
cudaError_t cudaMemsetAsync(void *d, int v, size_t n, cudaStream_t) { std::memset(d, v, n); return cudaSuccess; }
cudaError_t cudaStreamCreateWithFlags(cudaStream_t *s, unsigned) {
  *s = reinterpret_cast<cudaStream_t>(new int(0));
  return cudaSuccess;
}
cudaError_t cudaStreamDestroy(cudaStream_t s) { delete reinterpret_cast<int *>(s); return cudaSuccess; }
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaEventCreateWithFlags(cudaEvent_t *e, unsigned) {
  *e = reinterpret_cast<cudaEvent_t>(new FakeEvent{0, 0});
  return cudaSuccess;
}
cudaError_t cudaEventDestroy(cudaEvent_t e) { delete reinterpret_cast<FakeEvent *>(e); return cudaSuccess; }
cudaError_t cudaEventRecord(cudaEvent_t e, cudaStream_t) {
  std::lock_guard<std::mutex> lk(g_mu);
  reinterpret_cast<FakeEvent *>(e)->remaining = g_event_delay.load();
  reinterpret_cast<FakeEvent *>(e)->epoch = g_epoch.load();
  return cudaSuccess;
}
cudaError_t cudaEventSynchronize(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaEventCreate(cudaEvent_t *e) { return cudaEventCreateWithFlags(e, 0); }
cudaError_t cudaEventElapsedTime(float *ms, cudaEvent_t, cudaEvent_t) { *ms = 0.25f; return cudaSuccess; }
cudaError_t cudaStreamWaitEvent(cudaStream_t, cudaEvent_t, unsigned) { return cudaSuccess; }
cudaError_t cudaEventQuery(cudaEvent_t e) {
  auto *f = reinterpret_cast<FakeEvent *>(e);
  std::lock_guard<std::mutex> lk(g_mu);
  if (f->epoch < g_epoch.load()) return cudaSuccess;
  if (f->remaining > 0) { f->remaining--; return cudaErrorNotReady; }
  return cudaSuccess;
}
}  // extern "C"

namespace hk {

// With the shared background (Request::sym): the completion counters and fixed-point sums start
// at zero, and the far/near plan of every row tile (SymPlan, as the kernels compute it from
// the set's time table, far and shared near tiles) covers every ordered block (rows of column
// tile H, columns of column tile J) at most once, and exactly once where a term can be nonzero (J
// inside the window of H's row tile, and, for a later J, H inside the window of J's row tile), at
// the launch's plan level and at the other one; e_col(I) counts the far column tiles of later row
// tiles that hold I's columns.
static bool sym_fail(const char *what, int a, int b, int c) {
  std::fprintf(stderr, "symmetric plan check failed: %s (%d, %d, %d)\n", what, a, b, c);
  return false;
}

static bool check_plan_coverage(const Request &R);

static bool check_symmetry(const Request &R) {
  const SetView &S = R.set;
  if (!R.rt_done || !R.fixsum || S.win32.nb == 0) return sym_fail("set-up", S.n, 0, 0);
  for (int s = 0; s < num_sums(R.grad != 0, R.mix); ++s)  // the far pass scales by a float 2^F
    if (R.fix_bits[s] < -100 || R.fix_bits[s] > 120 || (s == 0 && R.fix_bits[0] > 126)) return sym_fail("fix_bits", S.n, s, R.fix_bits[s]);
  for (int I = 0; I < S.nrt; ++I)
    if (R.rt_done[I] != 0u) return sym_fail("rt_done not zero", S.n, I, 0);
  for (size_t i = 0; i < (size_t)num_sums(R.grad != 0, R.mix) * S.npad; ++i)
    if (R.fixsum[i] != 0) return sym_fail("fixsum not zero", S.n, (int)i, 0);
  if (R.sym != (HK_SYM_NEAR ? 2 : 1)) return sym_fail("level", S.n, R.sym, R.mix);
  if (S.nct > 1024) return true;  // the block table below grows as nct^2
  g_sym_checked++;
  // the launch's own plan level, then the other one (the build switch HK_SYM_NEAR picks between
  // them), on the same set and reaches
  Request other = R;
  other.sym = 3 - R.sym;
  return check_plan_coverage(R) && check_plan_coverage(other);
}

// Block coverage of one request's plan (SymPlan at its level R.sym) over its set.
static bool check_plan_coverage(const Request &R) {
  const SetView &S = R.set;
  auto tfirst = [&](int K) { return (double)S.t32[(size_t)K * kRowTile]; };
  std::vector<int2> win(S.nrt);
  std::vector<SymPlan> plan(S.nrt);
  for (int I = 0; I < S.nrt; ++I) {
    const int r1 = std::min((I + 1) * kRowTile, S.n) - 1;
    win[I] = table_window(S.win32, S.n, S.nct, tfirst(I) - R.cut_early, (double)S.t32[r1] + R.cut_late);
    plan[I] = sym_plan_scan(R, S.win32, I, win[I], tfirst);
    const int real = (S.n + kColTile - 1) / kColTile;  // column tiles holding real events
    if (plan[I].sym_end < win[I].x || plan[I].sym_end > 2 * I || plan[I].end < std::min(2 * I + 2, real) ||
        plan[I].end > win[I].y || plan[I].near_end < plan[I].sym_end || plan[I].near_end > 2 * I ||
        (R.sym != 2 && plan[I].near_end != plan[I].sym_end))
      return sym_fail("plan bounds", S.n, I, plan[I].sym_end * 10000 + plan[I].end);
  }
  const size_t nct = (size_t)S.nct;
  std::vector<int> cov(nct * nct, 0), ecol(S.nrt, 0);
  for (int I = 0; I < S.nrt; ++I)
    for (int J = win[I].x; J < plan[I].end; ++J) {  // row side: every column tile of I's window
      cov[(size_t)(2 * I) * nct + J]++;
      cov[(size_t)(2 * I + 1) * nct + J]++;
    }
  for (int K = 0; K < S.nrt; ++K)
    for (int H = win[K].x; H < plan[K].near_end; ++H) {  // column side of K's far and shared near tiles
      cov[(size_t)H * nct + 2 * K]++;
      cov[(size_t)H * nct + 2 * K + 1]++;
      if (H < plan[K].sym_end) ecol[H / 2]++;
    }
  for (int I = 0; I < S.nrt; ++I)
    if (ecol[I] != plan[I].e_col) return sym_fail("e_col", S.n, I, ecol[I] * 10000 + plan[I].e_col);
  for (int H = 0; H < S.nct; ++H)
    for (int J = 0; J < S.nct; ++J) {
      const int c = cov[(size_t)H * nct + J];
      const int I = H / 2, IJ = J / 2;
      const bool need = J >= win[I].x && J < win[I].y && (J <= H || (H >= win[IJ].x && H < win[IJ].y));
      if (c > 1 || (need && c != 1)) return sym_fail("coverage", S.n, H, J * 10 + c);
    }
  return true;
}

// Check one request's work decomposition against its set.
static void check_schedule(const Request &R, int mode) {
  const SetView &S = R.set;
  // the float64 kernel's slices may cut column tiles into chunks
  bool ok = R.slices >= 1 && R.slices <= S.nct * (mode == 0 ? fp64_chunks_per_tile() : 1);
  // the launch tiers: 4-leaf items, then 2-leaf, then 1-leaf (mixed); 1-leaf only (float64)
  if (R.wide < 0 || R.wide > R.coarse || R.coarse > S.nrt || (mode == 0 && R.coarse != 0)) ok = false;
  // the launch order covers every (row tile, leaf) exactly once; an item's slot is its number,
  // and a row tile's items are consecutive, so base + node = p
  std::vector<char> seen((size_t)S.nrt * R.slices, 0);
  for (int p = 0; ok && p < pair_items(R); ++p) {
    const PairItem it = item_at(R, p);
    if (it.rt < 0 || it.rt >= S.nrt || it.node < 0 || it.base + it.node != p || it.base < 0) { ok = false; break; }
    if (it.span != 1 && it.span != 2 && it.span != 4) { ok = false; break; }
    if (first_item_of(R, it.rt) != it.base) { ok = false; break; }  // the inverse of the launch order
    const int l0 = it.node * it.span, l1 = std::min(l0 + it.span, R.slices);
    if (l0 >= R.slices) { ok = false; break; }
    for (int l = l0; l < l1; ++l)
      if (seen[(size_t)it.rt * R.slices + l]++) ok = false;
  }
  for (size_t i = 0; ok && i < seen.size(); ++i)
    if (seen[i] != 1) ok = false;
  if (S.npad != S.nrt * kRowTile || S.nct * kColTile != S.npad || S.n > S.npad || S.n < 1) ok = false;
  if (!(R.cut_early > 0.0) || !(R.cut_late > 0.0)) ok = false;
  if (!R.partials || !R.comp || !R.rt_sum || !R.rt_count || !R.out || !R.status) ok = false;
  for (int i = 0; ok && i < request_counters(R); ++i)
    if (R.rt_count[i] != 0u) ok = false;  // merge-tree and completion counters zeroed before the launch
  if (ok && R.sym) ok = check_symmetry(R);
  if (ok && R.fixsum && !R.sym) {  // a grouped batch's fixed-point sums: zeroed, scales in range
    for (int s = 0; ok && s < num_sums(R.grad != 0, R.mix); ++s) ok = R.fix_bits[s] >= -100 && R.fix_bits[s] <= 120;
    for (int I = 0; ok && I < S.nrt; ++I) ok = R.rt_done[I] == 0u;
    for (size_t i = 0; ok && i < (size_t)num_sums(R.grad != 0, R.mix) * S.npad; ++i) ok = R.fixsum[i] == 0;
  }
  if (!ok) g_schedule_errors++;
}

// Output of a request: a function of its own inputs only, so the tests can tell where it went.
static void fake_outputs(const Batch &b, bool grad) {
  for (int r = 0; r < b.nreq; ++r) {
    const Request &R = b.req[r];
    if (grad && (R.flags & kFlagTestWithholdReady)) {  // the kernels' merge wait ran out
      if (R.status) *R.status |= kStatusMergeTimeout;
      for (int q = 0; q < 7; ++q) R.out[q] = std::nan("");
      continue;
    }
    R.out[0] = R.mu0 * 1000.0 + R.set.n + (b.mode ? 0.5 : 0.0) + (R.mix > 1 ? 0.25 : 0.0);
    if (grad) {
      const double th[9] = {R.mu0, R.tau_x, R.tau_t, R.theta, R.omega, R.h,
                            b.mix2.theta2, b.mix2.omega2, b.mix2.h2};
      for (int q = 0; q < (R.mix > 1 ? 9 : 6); ++q) R.out[1 + q] = th[q];
    }
    if (R.mu_out)
      for (int i = 0; i < R.set.n; ++i) { R.mu_out[i] = i; R.xi_out[i] = -i; }
    if (R.pi_out)
      for (int i = 0; i < R.set.n; ++i) R.pi_out[i] = R.mu0 + i;
  }
}

static cudaError_t fake_pair(const Batch &b, bool grad) {
  g_launches++;
  int items = 0;
  if (b.group) {  // grouped kernel: compensator items, then one item per (group, row tile, slice)
    for (int r = 0; r < b.nreq; ++r) {
      items += comp_items(b.req[r]);
      check_schedule(b.req[r], b.mode);
      const Request &R = b.req[r], &L = b.req[0];
      if (R.set.x32 != L.set.x32 || R.slices != L.slices || R.flags != L.flags || R.tscale != 1.0)
        g_schedule_errors++;  // one set, one decomposition, raw-unit moments
    }
    if (items != b.comp_total || b.mode != 1) g_schedule_errors++;
    for (int r = 0; r < b.nreq; ++r)  // every request of a grouped batch in fixed point, or none
      if ((b.req[r].fixsum != nullptr) != (b.req[0].fixsum != nullptr) || b.req[r].sym) g_schedule_errors++;
    items += (b.nreq + b.group - 1) / b.group * pair_items(b.req[0]);
  } else {
    for (int r = 0; r < b.nreq; ++r) {
      if (b.req[r].item_begin != items) g_schedule_errors++;
      if (b.req[r].sym && !b.split) g_schedule_errors++;  // sym rows are finished by the split epilogue
      items += request_items(b.req[r]);
      check_schedule(b.req[r], b.mode);
      // every pair item's partial-sum slot (num_sums doubles per row of the tile) lies before the
      // compensator sums, which the workspace places right after the slots
      const Request &R = b.req[r];
      // (none with the shared background, whose sums go to fixsum)
      const size_t slots = R.sym ? 0 : (size_t)pair_items(R) * num_sums(R.grad != 0, R.mix) * kRowTile;
      if (R.partials + slots > R.comp) g_schedule_errors++;
    }
  }
  if (items != b.total_items || !b.fused) g_schedule_errors++;
  fake_outputs(b, grad);
  return cudaSuccess;
}

// CPU model of the upload preparation launch (upload.cu): float32 copies, padding, tie
// indices, window tables and the input checks, on the fake runtime's host memory.
cudaError_t launch_upload_prep(const UploadPrep &u, cudaStream_t) {
  if (u.n < 1 || u.npad < u.n) return cudaErrorInvalidValue;
  unsigned flag = 0;
  const double tn = u.st[u.n - 1];
  int64_t s64 = 0, s32 = 0;
  for (int64_t i = 0; i < u.npad; ++i) {
    if (i < u.n) {
      const double x = u.sx[i], y = u.sy[i], t = u.st[i];
      if (!(std::fabs(x) <= 1e30) || !(std::fabs(y) <= 1e30) || !(t >= 0.0 && t <= 1e30)) flag |= 1u;
      if (i > 0 && !(t >= u.st[i - 1])) flag |= 2u;
      u.x64[i] = x; u.y64[i] = y; u.t64[i] = t;
      u.x32[i] = (float)x; u.y32[i] = (float)y; u.t32[i] = (float)t;
      if (i > 0 && u.st[i] != u.st[i - 1]) s64 = i;
      if (i > 0 && (float)u.st[i] != (float)u.st[i - 1]) s32 = i;
      u.lo64[i] = (int)s64; u.lo32[i] = (int)s32;
    } else {
      u.x64[i] = 0.0; u.y64[i] = 0.0; u.t64[i] = tn;
      u.x32[i] = 0.f; u.y32[i] = 0.f; u.t32[i] = (float)tn;
      u.lo64[i] = u.lo32[i] = (int)u.n;
    }
  }
  const int nb = kWinBuckets, real = (int)((u.n + kColTile - 1) / kColTile);
  for (int f64 = 0; f64 < 2; ++f64) {
    int *w = f64 ? u.w64 : u.w32;
    if (!w) continue;
    const double t0 = f64 ? u.t0_64 : u.t0_32, width = f64 ? u.width_64 : u.width_32;
    auto tm = [&](int64_t j) { return f64 ? u.st[j] : (double)(float)u.st[j]; };
    int c = 0;
    for (int b = 0; b < nb; ++b) {
      const double lo = t0 + (double)b * width;
      while (c < real && tm(std::min<int64_t>((int64_t)(c + 1) * kColTile, u.n) - 1) < lo) ++c;
      w[b] = c;
    }
    c = 0;
    for (int b = 0; b < nb; ++b) {
      const double hi = t0 + (double)(b + 1) * width;
      while (c < real && tm((int64_t)c * kColTile) <= hi) ++c;
      w[nb + b] = c;
    }
  }
  *u.flags |= flag;
  return cudaSuccess;
}

cudaError_t launch_pair_mixed(const Batch &b, bool grad, cudaStream_t) { return fake_pair(b, grad); }
// The split epilogue: fake_pair already wrote every output; count the launch and check that it
// follows a split mixed-precision batch.
cudaError_t init_log_table() { return cudaSuccess; }
cudaError_t launch_epilogue_fix(const Batch &b, bool, cudaStream_t) {
  if (!b.split || b.mode != 1 || b.group) g_schedule_errors++;
  return cudaSuccess;
}
cudaError_t launch_pair_fp64(const Batch &b, bool grad, cudaStream_t) { return fake_pair(b, grad); }
cudaError_t launch_pair_group(const Batch &b, bool grad, cudaStream_t) {
  // the group size the host picked for this batch, and one the kernel is built for
  bool built = false;
  if (grad) {
    for (int G : kGroupSizesGrad) built |= b.group == G;
  } else {
    for (int G : kGroupSizesLoglik) built |= b.group == G;
  }
  if (!built || b.group != group_size(grad, b.nreq)) g_schedule_errors++;
  g_last_group = b.group;
  g_group_launches++;
  return fake_pair(b, grad);
}

int fp64_chunks_per_tile() { return 8; }

int occupancy_pair_mixed(bool) { return 4; }
int occupancy_pair_fp64(bool) { return 2; }

}  // namespace hk
