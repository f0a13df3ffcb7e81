// Unit probes for the roofline and the accuracy analysis of the mixed-precision path.
//
// 1. Issue rate of the float32 pipe: packed FFMA2, FADD2 and FMUL2, unpacked FFMA and FADD, a
//    packed FADD2 + FFMA2 mix, MUFU.EX2 (ex2.approx.ftz.f32), and half the chains packed FFMA2
//    with the other half scalar FFMA (whether the two share one pipe), each over 8 independent chains
//    per thread, 4 CTAs of 256 threads per SM; lane operations per second from CUDA events.
// 2. Mean and RMS relative error of ex2.approx.ftz.f32 against exp2 in double, for arguments
//    -q with q drawn uniformly from each quarter-unit bin of [0, 16): the argument-dependent
//    bias of the float32 exponential that the pair kernels use.
// 3. Rates of the float64 and conversion sequences that accumulate the row sums (see
//    rate64_kernel), in sequences per second.
// Prints one JSON object. Built and run by bench.py --probe-units.
#include <cmath>
#include <cstdio>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ float ex2a(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr int kChains = 8, kIters = 4096;

template <int OP>
__global__ void rate_kernel(float *out, float s) {
  float2 a[kChains];
  const float2 b = make_float2(s, s * 0.5f), one = make_float2(1.f, 1.f);
  for (int i = 0; i < kChains; ++i) a[i] = make_float2(threadIdx.x * 1e-9f + i, i * 0.5f);
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      if (OP == 0) a[i] = __ffma2_rn(a[i], b, b);
      if (OP == 1) a[i] = __fadd2_rn(a[i], b);
      if (OP == 2) a[i] = __fmul2_rn(a[i], b);
      if (OP == 3) { a[i].x = __fmaf_rn(a[i].x, b.x, b.y); a[i].y = __fmaf_rn(a[i].y, b.x, b.y); }
      if (OP == 4) { a[i].x = __fadd_rn(a[i].x, b.x); a[i].y = __fadd_rn(a[i].y, b.x); }
      if (OP == 5) { a[i] = __fadd2_rn(a[i], b); a[i] = __ffma2_rn(a[i], b, one); }
      if (OP == 6) a[i].x = ex2a(a[i].x);
      if (OP == 7) {  // half the chains packed FFMA2, half two scalar FFMA
        if (i < kChains / 2) a[i] = __ffma2_rn(a[i], b, b);
        else { a[i].x = __fmaf_rn(a[i].x, b.x, b.y); a[i].y = __fmaf_rn(a[i].y, b.x, b.y); }
      }
    }
  }
  float acc = 0.f;
  for (int i = 0; i < kChains; ++i) acc += a[i].x + a[i].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

template <int OP>
double lane_ops_per_s(int sms, double lanes_per_iter_and_chain) {
  const int threads = 256, blocks = sms * 4;
  float *out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(float)) != cudaSuccess) return -1.0;
  rate_kernel<OP><<<blocks, threads>>>(out, 1.0001f);  // warm-up
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(e0);
    rate_kernel<OP><<<blocks, threads>>>(out, 1.0001f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return (double)blocks * threads * kIters * kChains * lanes_per_iter_and_chain / (best * 1e-3);
}

// Float64 and conversion rates, one dependent chain per (thread, chain), the same launch shape:
// 7 DADD; 8 a float32 value folded into a float64 sum (FMUL, F2F.F64.F32, DADD); 9 a float32
// value into an int64 sum (FMUL, F2I.S64.F32, 64-bit add); 10 a double into an int64 sum (DMUL,
// F2I.S64.F64, 64-bit add); 12 log of a double (CUDA's log) and an add; 13 the correctly
// rounded float64 reciprocal and an add; 14 a float64 division and an add.
template <int OP>
__global__ void rate64_kernel(float *out, float s) {
  double d[kChains];
  float f[kChains];
  long long l[kChains];
  const double c = 1.0000001 + (double)s * 1e-9;
  for (int i = 0; i < kChains; ++i) {
    d[i] = threadIdx.x * 1e-9 + i;
    f[i] = 1.0f + i * 0.25f;
    l[i] = threadIdx.x + i;
  }
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      if (OP == 7) d[i] = __dadd_rn(d[i], c);
      if (OP == 8) { f[i] = __fmul_rn(f[i], s); d[i] = __dadd_rn(d[i], (double)f[i]); }
      if (OP == 9) { f[i] = __fmul_rn(f[i], s); l[i] += __float2ll_rn(f[i]); }
      if (OP == 10) { d[i] = __dmul_rn(d[i], c); l[i] += __double2ll_rn(d[i]); }
      if (OP == 12) d[i] = log(d[i]) + 3.0;
      if (OP == 13) d[i] = __drcp_rn(d[i]) + 3.0;
      if (OP == 14) d[i] = 1.0 / d[i] + 3.0;
    }
  }
  double acc = 0.0;
  for (int i = 0; i < kChains; ++i) acc += d[i] + f[i] + (double)l[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)acc;
}

template <int OP>
double ops64_per_s(int sms) {
  const int threads = 256, blocks = sms * 4;
  float *out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(float)) != cudaSuccess) return -1.0;
  rate64_kernel<OP><<<blocks, threads>>>(out, 1.0001f);  // warm-up
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    rate64_kernel<OP><<<blocks, threads>>>(out, 1.0001f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return (double)blocks * threads * kIters * kChains / (best * 1e-3);
}

constexpr int kBins = 64;  // q in [0, 16), bins of 0.25

__global__ void ex2_error_kernel(unsigned long long seed, double *sum, double *sum2, unsigned long long *cnt) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x, bin = gid % kBins;
  unsigned long long st = seed + (unsigned long long)gid * 0x9E3779B97F4A7C15ull;
  double a1 = 0.0, a2 = 0.0;
  for (int it = 0; it < 512; ++it) {
    st ^= st << 13;
    st ^= st >> 7;
    st ^= st << 17;
    const float q = (float)((bin + (double)(st >> 11) * (1.0 / 9007199254740992.0)) * 0.25);
    const double r = (double)ex2a(-q) / exp2(-(double)q) - 1.0;
    a1 += r;
    a2 += r * r;
  }
  atomicAdd(&sum[bin], a1);
  atomicAdd(&sum2[bin], a2);
  atomicAdd(&cnt[bin], 512ull);
}

}  // namespace

int main() {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) return 1;
  std::printf("{\"sms\": %d, \"lane_ops_per_s\": {", sms);
  std::printf("\"ffma2\": %.6e, ", lane_ops_per_s<0>(sms, 2.0));
  std::printf("\"fadd2\": %.6e, ", lane_ops_per_s<1>(sms, 2.0));
  std::printf("\"fmul2\": %.6e, ", lane_ops_per_s<2>(sms, 2.0));
  std::printf("\"ffma\": %.6e, ", lane_ops_per_s<3>(sms, 2.0));
  std::printf("\"fadd\": %.6e, ", lane_ops_per_s<4>(sms, 2.0));
  std::printf("\"fadd2_ffma2\": %.6e, ", lane_ops_per_s<5>(sms, 4.0));
  std::printf("\"mufu_ex2\": %.6e, ", lane_ops_per_s<6>(sms, 1.0));
  std::printf("\"ffma2_ffma_mix\": %.6e}, ", lane_ops_per_s<7>(sms, 2.0));
  std::printf("\"sequences_per_s\": {");
  std::printf("\"dadd\": %.6e, ", ops64_per_s<7>(sms));
  std::printf("\"fold_f32_into_f64\": %.6e, ", ops64_per_s<8>(sms));
  std::printf("\"f32_into_int64\": %.6e, ", ops64_per_s<9>(sms));
  std::printf("\"f64_into_int64\": %.6e, ", ops64_per_s<10>(sms));
  std::printf("\"log_f64\": %.6e, ", ops64_per_s<12>(sms));
  std::printf("\"rcp_rn_f64\": %.6e, ", ops64_per_s<13>(sms));
  std::printf("\"div_f64\": %.6e}, ", ops64_per_s<14>(sms));
  double *s1 = nullptr, *s2 = nullptr;
  unsigned long long *c = nullptr;
  if (cudaMalloc(&s1, kBins * 8) != cudaSuccess || cudaMalloc(&s2, kBins * 8) != cudaSuccess ||
      cudaMalloc(&c, kBins * 8) != cudaSuccess)
    return 1;
  cudaMemset(s1, 0, kBins * 8);
  cudaMemset(s2, 0, kBins * 8);
  cudaMemset(c, 0, kBins * 8);
  ex2_error_kernel<<<1024, 256>>>(12345ull, s1, s2, c);
  double h1[kBins], h2[kBins];
  unsigned long long hc[kBins];
  cudaMemcpy(h1, s1, sizeof(h1), cudaMemcpyDeviceToHost);
  cudaMemcpy(h2, s2, sizeof(h2), cudaMemcpyDeviceToHost);
  cudaMemcpy(hc, c, sizeof(hc), cudaMemcpyDeviceToHost);
  std::printf("\"ex2_rel_err\": {\"bin_width\": 0.25, \"mean\": [");
  for (int b = 0; b < kBins; ++b) std::printf("%s%.4e", b ? ", " : "", h1[b] / (double)hc[b]);
  std::printf("], \"rms\": [");
  for (int b = 0; b < kBins; ++b) std::printf("%s%.4e", b ? ", " : "", std::sqrt(h2[b] / (double)hc[b]));
  std::printf("]}}\n");
  cudaFree(s1);
  cudaFree(s2);
  cudaFree(c);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
