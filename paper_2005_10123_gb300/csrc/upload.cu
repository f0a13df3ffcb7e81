// Upload preparation on the device: two launches turn the caller's float64 coordinates into
// everything the pair kernels read (SetView): the float64 and float32 copies, the padding,
// the tie indices lo and the two column-tile time tables (WinTable), and check the inputs on
// the way. The coordinates are read from sx, sy, st: the caller's host arrays themselves where
// the device can read pageable host memory, else the set's own x64, y64, t64 after a copy.
//
// Pass 1 (upload_events_kernel), one coalesced pass over the source arrays, grid-stride over
// the padded length:
//   i < n:  x64, y64, t64 copied; x32, y32, t32 = the float64 values rounded to nearest; flag 1
//           if a coordinate is not finite within 1e30 or a time is outside [0, 1e30], flag 2 if
//           t_i < t_{i-1};
//   i >= n: coordinates 0 and the time t_N (the kernels substitute a sentinel for padded
//           events).
// Pass 2 (upload_index_kernel), over the copies pass 1 wrote (device memory, so the searches
// below never wait on host memory):
//   lo[i] = the first index whose stored time equals t_i (Section 2.1's strict indicator
//           t_n' < t_n is n' < lo[n] for sorted times), from the float64 times for lo64 and
//           from their float32 roundings for lo32; lo = n for padded events;
//   tables, one thread per entry: for bucket b of width w from t0, first[b] = the number of
//           column tiles whose latest time is below t0 + b w and last[b] = the number of column
//           tiles whose earliest time is at most t0 + (b + 1) w, by binary search over the tiles
//           (the times ascend). Bucket edges are formed without fused multiply-add so that they
//           are the same on every build.
// One pass did everything before, its searches reading the caller's host memory: 0.060 ms for
// an 85,000-event upload (host-timed call) against 0.050 ms now.
// For decreasing or non-finite times the indices and tables are meaningless, and the host
// rejects the set from the flags.
#include "upload.h"

namespace hk {
namespace {

constexpr int kPrepThreads = 256;

// First index j in [0, i] whose value equals v_i, for values that ascend up to i.
template <typename F>
__device__ __forceinline__ int tie_start(F get, int64_t i) {
  const auto v = get(i);
  if (i == 0 || get(i - 1) != v) return (int)i;
  int64_t a = 0, b = i - 1;  // get(b) == v: find the first such index
  while (a < b) {
    const int64_t m = (a + b) / 2;
    if (get(m) < v) a = m + 1;
    else b = m;
  }
  return (int)a;
}

// Pass 1, events: the one pass over the caller's arrays (host memory the device reads in place,
// or the set's own float64 copy), coalesced, one event per thread: the float64 and float32
// copies, the padding and the checks. The tie indices and tables come in pass 2 from the copies
// this pass writes, so that no search runs over host memory.
__global__ void __launch_bounds__(kPrepThreads) upload_events_kernel(const UploadPrep u) {
  unsigned flag = 0;
  const double tn = u.st[u.n - 1];
  const int64_t stride = (int64_t)gridDim.x * kPrepThreads;
  for (int64_t i = (int64_t)blockIdx.x * kPrepThreads + threadIdx.x; i < u.npad; i += stride) {
    if (i < u.n) {
      const double x = u.sx[i], y = u.sy[i], t = u.st[i];
      if (!(fabs(x) <= 1e30) || !(fabs(y) <= 1e30) || !(t >= 0.0 && t <= 1e30)) flag |= 1u;
      if (i > 0 && !(t >= u.st[i - 1])) flag |= 2u;
      u.x64[i] = x;
      u.y64[i] = y;
      u.t64[i] = t;
      u.x32[i] = __double2float_rn(x);
      u.y32[i] = __double2float_rn(y);
      u.t32[i] = __double2float_rn(t);
    } else {
      u.x64[i] = 0.0;
      u.y64[i] = 0.0;
      u.t64[i] = tn;
      u.x32[i] = 0.f;
      u.y32[i] = 0.f;
      u.t32[i] = __double2float_rn(tn);
    }
  }
  flag = __reduce_or_sync(0xffffffffu, flag);
  if ((threadIdx.x & 31) == 0 && flag) atomicOr(u.flags, flag);
}

// Pass 2, over the device copies of pass 1: the tie indices (blocks [0, event_blocks)) and the
// window tables (the blocks after them).
__global__ void __launch_bounds__(kPrepThreads) upload_index_kernel(const UploadPrep u, int event_blocks) {
  if ((int)blockIdx.x < event_blocks) {
    auto t64 = [&](int64_t j) { return u.t64[j]; };
    auto t32 = [&](int64_t j) { return u.t32[j]; };
    const int64_t stride = (int64_t)event_blocks * kPrepThreads;
    for (int64_t i = (int64_t)blockIdx.x * kPrepThreads + threadIdx.x; i < u.npad; i += stride) {
      if (i < u.n) {
        u.lo64[i] = tie_start(t64, i);
        u.lo32[i] = tie_start(t32, i);
      } else {
        u.lo64[i] = (int)u.n;
        u.lo32[i] = (int)u.n;
      }
    }
    return;
  }
  const int q = ((int)blockIdx.x - event_blocks) * kPrepThreads + (int)threadIdx.x;
  const int nb = kWinBuckets;
  if (q >= 4 * nb) return;
  const bool f64 = q >= 2 * nb, upper = (q % (2 * nb)) >= nb;
  const int b = q % nb;
  int *w = f64 ? u.w64 : u.w32;
  if (!w) return;  // no table for these times
  const double t0 = f64 ? u.t0_64 : u.t0_32, width = f64 ? u.width_64 : u.width_32;
  auto tm = [&](int64_t j) { return f64 ? u.t64[j] : (double)u.t32[j]; };
  const int real = (int)((u.n + kColTile - 1) / kColTile);  // column tiles holding real events
  int a = 0, e = real;
  if (!upper) {  // first tile whose latest time is >= the bucket's start
    const double lo = __dadd_rn(t0, __dmul_rn((double)b, width));
    while (a < e) {
      const int m = (a + e) / 2;
      const int64_t last = ((int64_t)m + 1) * kColTile < u.n ? ((int64_t)m + 1) * kColTile - 1 : u.n - 1;
      if (tm(last) < lo) a = m + 1;
      else e = m;
    }
    w[b] = a;
  } else {  // first tile whose earliest time is > the bucket's end
    const double hi = __dadd_rn(t0, __dmul_rn((double)(b + 1), width));
    while (a < e) {
      const int m = (a + e) / 2;
      if (tm((int64_t)m * kColTile) <= hi) a = m + 1;
      else e = m;
    }
    w[nb + b] = a;
  }
}

}  // namespace

cudaError_t launch_upload_prep(const UploadPrep &u, cudaStream_t s) {
  if (u.n < 1 || u.npad < u.n) return cudaErrorInvalidValue;
  const int64_t need = (u.npad + kPrepThreads - 1) / kPrepThreads, cap = (int64_t)(u.sms > 0 ? u.sms : 1) * 8;
  const int event_blocks = (int)(need < cap ? need : cap);
  const int table_blocks = (4 * kWinBuckets + kPrepThreads - 1) / kPrepThreads;
  upload_events_kernel<<<event_blocks, kPrepThreads, 0, s>>>(u);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  upload_index_kernel<<<event_blocks + table_blocks, kPrepThreads, 0, s>>>(u, event_blocks);
  return cudaGetLastError();
}

}  // namespace hk
