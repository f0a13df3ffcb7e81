// hawkes_loglik_noalloc: the mixed-precision log-likelihood for callers that cannot
// allocate device memory.
//
// Who needs it: code that may not call cudaMalloc/cudaFree at evaluation time, for
// example a host program whose device memory is entirely reserved up front by another
// allocator (a framework's memory pool), or a latency-critical sampler loop in which an
// allocation or free could block on device-wide synchronisation. Such callers keep their
// events in device buffers they already own and pass those in; every temporary the
// evaluation needs lives in one file-scope device array, g_scratch, that the library
// reserves when it is loaded and keeps until the process exits (on every GPU that loads
// it, kScratchBytes each).
//
// The pair sums come from the library's ordinary mixed-precision pair kernel; this file
// prepares its inputs inside g_scratch (padded float32 copies, tie indices, input checks) with
// one small kernel and finishes with its own epilogue, which reads t_N from the device so that
// the whole call stays asynchronous. The inputs are never read on the host, so their checks run
// on the device: an input the context path would reject (unsorted, negative or non-finite
// times, non-finite coordinates, a scaled time span beyond float32's range) makes the result
// NaN.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/hawkes.h"
#include "hk_internal.h"

namespace hk {
namespace {

constexpr int kNoallocMax = HAWKES_NOALLOC_MAX_EVENTS;  // 65,536 events
constexpr int kChunks = 4;                               // most column chunks per row tile
constexpr int kMaxRowTiles = (kNoallocMax + kRowTile - 1) / kRowTile;
constexpr int kMaxItems = kMaxRowTiles * kChunks;

// Layout of g_scratch (byte offsets, all 256-aligned).
constexpr size_t kOffHeader = 0;  // 1 KB, zeroed by every call: epilogue ticket at +256, check flag at +512
constexpr size_t kOffTicket = kOffHeader + 256;
constexpr size_t kOffCheck = kOffHeader + 512;
constexpr size_t kOffX = 1024;
constexpr size_t kOffY = kOffX + (size_t)kNoallocMax * 4;
constexpr size_t kOffT = kOffY + (size_t)kNoallocMax * 4;
constexpr size_t kOffLo = kOffT + (size_t)kNoallocMax * 4;
constexpr size_t kOffBlockPart = kOffLo + (size_t)kNoallocMax * 4;
constexpr size_t kOffPartials = kOffBlockPart + (size_t)(kNoallocMax / kEpiThreads) * 8 * 8;
constexpr size_t kScratchBytes = kOffPartials + (size_t)kMaxItems * kSumsLoglik * kRowTile * 8;
static_assert(kOffBlockPart % 256 == 0 && kOffPartials % 256 == 0, "scratch regions must stay 256-byte aligned");

// The scratch array. In host code this name is only a stand-in symbol, not a device
// address: host code obtains the address with cudaGetSymbolAddress (see scratch_base).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Fill the padded float32 copies and the tie indices lo[i] (first index whose time equals
// t[i], by binary search; the search stays in [0, i] for any input), and check the inputs of
// Section 2.1's domain: finite coordinates, finite times >= 0 in non-decreasing order, and a
// scaled time span beta (t_N - t_1) below 1e15 (the float32 path's range). A failed check sets
// the check flag, and the epilogue then writes NaN.
__global__ void noalloc_prep(const float *__restrict__ x, const float *__restrict__ y,
                             const float *__restrict__ t, int n, int npad, double beta, unsigned char *scratch) {
  float *sx = (float *)(scratch + kOffX), *sy = (float *)(scratch + kOffY), *st = (float *)(scratch + kOffT);
  int *lo = (int *)(scratch + kOffLo);
  unsigned *check = (unsigned *)(scratch + kOffCheck);
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += stride) {
    if (i < n) {
      const float ti = t[i], xi = x[i], yi = y[i];
      bool bad = !isfinite(xi) || !isfinite(yi) || !isfinite(ti) || ti < 0.f;
      if (i > 0) bad |= !(t[i - 1] <= ti);
      if (i == n - 1) bad |= !((double)ti - (double)t[0] <= 1.0e15 / beta);
      if (bad) atomicOr(check, 1u);
      sx[i] = xi;
      sy[i] = yi;
      st[i] = ti;
      int a = 0, b = i;  // first index in [0, i] whose time is >= t[i]
      while (a < b) {
        const int m = (a + b) >> 1;
        if (t[m] < ti) a = m + 1; else b = m;
      }
      lo[i] = a;
    } else {
      sx[i] = 0.f;
      sy[i] = 0.f;
      st[i] = t[n - 1];
      lo[i] = n;
    }
  }
}

// log lambda_n - Lambda_n per event and a fixed-order sum (warp tree, warps in order,
// blocks in order by the last block to finish), as the library's epilogue does, with
// t_N = t[n-1] taken from the float32 copy on the device. NaN if the input checks failed.
__global__ void __launch_bounds__(kEpiThreads) noalloc_epilogue(const __grid_constant__ Request R, int chunks,
                                                                unsigned char *scratch) {
  constexpr int NW = kEpiThreads / 32;
  __shared__ double red[NW];
  __shared__ int s_last;
  const float *st = (const float *)(scratch + kOffT);
  const double *partials = (const double *)(scratch + kOffPartials);
  double *block_part = (double *)(scratch + kOffBlockPart);
  unsigned *ticket = (unsigned *)(scratch + kOffTicket);
  const unsigned *check = (const unsigned *)(scratch + kOffCheck);
  const int n = R.set.n, nblk = (n + kEpiThreads - 1) / kEpiThreads;
  const double t_last = (double)st[n - 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int i = blk * kEpiThreads + tid;
    double v = 0.0;
    if (i < n) {
      const int rt = i / kRowTile, li = i - rt * kRowTile;
      double sb = 0.0, ss = 0.0;
      for (int c = 0; c < chunks; ++c) {
        const double *src = partials + (size_t)(rt * chunks + c) * kSumsLoglik * kRowTile + li;
        sb += src[0];
        ss += src[kRowTile];
      }
      const double A = R.mu0 * R.k_ab, C = R.theta * R.k_cw;
      const double tn = (double)st[i];
      const double Lam = R.mu0 * (normcdf((t_last - tn) * R.inv_tt) - normcdf(-tn * R.inv_tt)) +
                         R.theta * (1.0 - exp(-R.omega * (t_last - tn)));
      v = log(A * sb + C * ss) - Lam;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (tid == 0) {
      double x = 0.0;
#pragma unroll
      for (int w = 0; w < NW; ++w) x += red[w];
      block_part[blk] = x;
      __threadfence();
      s_last = (atomicAdd(ticket, 1u) == (unsigned)(nblk - 1));
    }
    __syncthreads();
    if (s_last) {  // fixed strided subsets, then a fixed-shape tree: deterministic
      __threadfence();
      double x = 0.0;
      for (int b = tid; b < nblk; b += kEpiThreads) x += __ldcg(block_part + b);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      __syncthreads();
      if (lane == 0) red[warp] = x;
      __syncthreads();
      if (tid == 0) {
        double y = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) y += red[w];
        R.out[0] = *check ? __longlong_as_double(0x7ff8000000000000ll) : y;
      }
    }
    __syncthreads();
  }
}

struct DeviceScratch {
  unsigned char *base = nullptr;
  int sms = 0;
  unsigned long long ctx_id = 0;  // the CUDA context the address belongs to
  bool ready = false;
};
constexpr int kMaxDevices = 64;
DeviceScratch g_dev[kMaxDevices];
std::mutex g_setup_mu;

// Identity of the calling thread's current CUDA context (driver entry points looked up once
// through the runtime, so the library does not link the driver library). A device reset
// (cudaDeviceReset) replaces the primary context and reloads the module, which can move
// g_scratch; a new context id makes scratch_base look the address up again.
using CtxGetCurrentFn = int (*)(void **);
using CtxGetIdFn = int (*)(void *, unsigned long long *);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

int current_ctx_id(unsigned long long *id) {
  *id = 0;
  if (!g_ctx_current || !g_ctx_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    void *f1 = nullptr, *f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess)
      return HAWKES_E_CUDA;
    g_ctx_current = (CtxGetCurrentFn)f1;
    g_ctx_id = (CtxGetIdFn)f2;
  }
  void *ctx = nullptr;
  if (g_ctx_current(&ctx) != 0) return HAWKES_E_CUDA;
  if (ctx && g_ctx_id(ctx, id) != 0) return HAWKES_E_CUDA;
  return HAWKES_OK;
}

// Set-up, with `device` current: the device address of g_scratch in the current context and the
// device's SM count. Done on the first call on each device (and again after the context changed).
int scratch_base(int device, DeviceScratch **out) {
  if (device < 0 || device >= kMaxDevices) return HAWKES_E_INVAL;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  DeviceScratch &d = g_dev[device];
  unsigned long long id = 0;
  if (int rc = current_ctx_id(&id)) return rc;
  if (!d.ready || id == 0 || id != d.ctx_id) {
    d.ready = false;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) return HAWKES_E_CUDA;
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return HAWKES_E_CUDA;
    if (int rc = current_ctx_id(&id)) return rc;  // the lookup made the primary context current
    if (id == 0) return HAWKES_E_CUDA;
    d.base = (unsigned char *)p;
    d.ctx_id = id;
    d.ready = true;
  }
  *out = &d;
  return HAWKES_OK;
}

}  // namespace
}  // namespace hk

using namespace hk;

extern "C" int hawkes_loglik_noalloc(const float *x, const float *y, const float *t, int64_t n,
                                     const hawkes_params *p, int flags, double *device_out,
                                     void *cuda_stream) {
  if (!x || !y || !t || !p || !device_out) return HAWKES_E_INVAL;
  if (n < 1 || n > kNoallocMax) return HAWKES_E_INVAL;  // above HAWKES_NOALLOC_MAX_EVENTS
  if (flags & ~(HAWKES_FLAG_EXCLUDE_SELF | HAWKES_FLAG_DENSE | HAWKES_FLAG_NO_SYMMETRY)) return HAWKES_E_INVAL;
  const double vals[6] = {p->mu0, p->tau_x, p->tau_t, p->theta, p->omega, p->h};
  for (int k = 0; k < 6; ++k)
    if (!std::isfinite(vals[k]) || (k == 3 ? vals[k] < 0.0 : vals[k] <= 0.0)) return HAWKES_E_INVAL;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return HAWKES_E_CUDA;
  DeviceScratch *d = nullptr;
  if (int rc = scratch_base(device, &d)) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int npad = (int)((n + kPadTo - 1) / kPadTo * kPadTo);
  const int nrt = npad / kRowTile, nct = npad / kColTile;
  const int chunks = std::min(kChunks, nct);
  unsigned char *base = d->base;

  // the request, exactly as the ordinary path describes a mixed loglik evaluation
  Batch b;
  std::memset(&b, 0, sizeof(b));
  b.nreq = 1;
  b.mode = 1;
  Request &R = b.req[0];
  R.set.x32 = (const float *)(base + kOffX);
  R.set.y32 = (const float *)(base + kOffY);
  R.set.t32 = (const float *)(base + kOffT);
  R.set.lo32 = (const int *)(base + kOffLo);
  R.set.n = (int)n; R.set.npad = npad; R.set.nrt = nrt; R.set.nct = nct;
  R.slices = chunks;
  R.grad = 0;
  R.flags = flags;
  const double log2e = 1.4426950408889634074;
  set_mixed_constants(&R, p->tau_x, p->tau_t, p->omega, p->h);
  if (!(R.a2 > 0.f) || !(R.beta > 0.f) || !(R.s_hi > 0.f) || !std::isfinite(R.a2) || !std::isfinite(R.wn) ||
      !(R.cn < 0.f) || !std::isfinite(R.cn))
    return HAWKES_E_INVAL;
  R.mu0 = p->mu0; R.tau_x = p->tau_x; R.tau_t = p->tau_t;
  R.theta = p->theta; R.omega = p->omega; R.h = p->h;
  {
    const double two_pi = 6.28318530717958647693;
    R.k_ab = 1.0 / (two_pi * std::sqrt(two_pi) * p->tau_x * p->tau_x * p->tau_t);
    R.k_cw = p->omega / (two_pi * p->h * p->h);
    R.inv_tx = 1.0 / p->tau_x; R.inv_tt = 1.0 / p->tau_t; R.inv_h = 1.0 / p->h; R.inv_om = 1.0 / p->omega;
  }
  // the exact-zero column window: every term that is not exactly zero in float32 (the context
  // path, with the self term, stops where all skipped terms of a row stay below 2^-40 of
  // lambda_n, see term_reaches there; the two agree to that bound)
  const double bg = 1.01 * std::sqrt(130.0) / (double)R.beta, trig = 1.01 * 131.0 / (p->omega * log2e);
  R.cut_early = std::max(bg, trig);
  R.cut_late = bg;
  R.comp = nullptr;  // noalloc_epilogue computes the compensator
  R.partials = (double *)(base + kOffPartials);
  R.out = device_out;
  R.t_last = 0.0;  // unused here: noalloc_epilogue reads t_N on the device

  // the epilogue ticket and the check flag must start at zero on every call
  if (cudaMemsetAsync(base + kOffHeader, 0, 1024, s) != cudaSuccess) return HAWKES_E_CUDA;
  noalloc_prep<<<std::min(d->sms * 4, (npad + 255) / 256 + 1), 256, 0, s>>>(x, y, t, (int)n, npad, 1.0 / R.tscale,
                                                                            base);
  if (cudaGetLastError() != cudaSuccess) return HAWKES_E_CUDA;
  b.req[0].item_begin = 0;
  b.total_items = nrt * chunks;
  b.fused = 0;  // noalloc_epilogue finishes the evaluation
  const int epi_blocks = (int)((n + kEpiThreads - 1) / kEpiThreads);
  if (launch_pair_mixed(b, false, s) != cudaSuccess) return HAWKES_E_CUDA;
  noalloc_epilogue<<<std::max(1, std::min(epi_blocks, d->sms * 8)), kEpiThreads, 0, s>>>(b.req[0], chunks,
                                                                                       base);
  if (cudaGetLastError() != cudaSuccess) return HAWKES_E_CUDA;
  return HAWKES_OK;
}
