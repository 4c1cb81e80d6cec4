// Roofline denominators measured on the running device (peak_probe in include/avip.h).  The
// paper has no counterpart: these are measurement aids for the benchmark, which reports each
// solver kernel against the rate this device reaches on the unit that bounds it.
//
//   FP64 FMA: every thread runs 8 independent chains a = a * m + c (no dependence between the
//             chains, so the FP64 pipe can issue every cycle it is free); 2 flops per FMA.
//   HBM copy: a grid-stride copy of 1 GiB in 16-byte vectors between two fresh buffers (each
//             far larger than the 129 MB L2); read + write bytes counted.
// Each figure is the best of several launches timed with CUDA events on the given stream,
// after one untimed launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "avip_internal.h"
#include "fp64_math.cuh"

namespace avip {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kFmaIters = 4096;
constexpr int kChains = 8;
constexpr size_t kCopyBytes = size_t(1) << 30;
constexpr int kTimedLaunches = 5;

__global__ void __launch_bounds__(kProbeThreads) fp64_fma_probe_kernel(double* out, double m, double c) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(kProbeThreads) copy_probe_kernel(const int4* __restrict__ src, int4* __restrict__ dst,
                                                                   size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = __ldcs(src + i);
}

// Best time (ms) of kTimedLaunches launches of `launch` after one untimed one.
template <typename F>
cudaError_t best_ms(cudaStream_t st, F launch, float& best) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch();
  best = 0.f;
  for (int k = 0; k < kTimedLaunches && e == cudaSuccess; ++k) {
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (k == 0 || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

// Largest relative difference between this library's FP64 exp / log / pow / reciprocal
// (fp64_math.cuh) and the CUDA math library (the IEEE quotient for the reciprocal) over
// log-spaced arguments: exp on [-700, 700], log on 1e-300 .. 1e300, pow (exponents -0.2, 0.5,
// -1.7, 2.3) on bases 1e-6 .. 1e6, the reciprocal on +-(1e-300 .. 1e300).
constexpr int kCheckPoints = 1 << 16;
__global__ void fp64_math_check_kernel(unsigned long long* worst) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kCheckPoints) return;
  const double t = (double)k / (kCheckPoints - 1);
  const double xe = -700.0 + 1400.0 * t;
  const double xl = exp10(-300.0 + 600.0 * t) * (1.0 + 0.3 * sin(37.0 * k));
  auto rel = [](double a, double b) { return b != 0.0 ? fabs(a - b) / fabs(b) : fabs(a); };
  double e[4];
  e[0] = rel(exp_fp64(xe), exp(xe));
  e[1] = rel(log_fp64(xl), log(xl));
  e[2] = 0.0;
  const double xr = (k & 1 ? -1.0 : 1.0) * xl;
  e[3] = rel(recip_nr(xr), 1.0 / xr);
  const double ps[4] = {-0.2, 0.5, -1.7, 2.3};
  for (double pp : ps) {
    const double xb = exp10(-6.0 + 12.0 * t) * (1.0 + 0.3 * sin(11.0 * k));
    e[2] = fmax(e[2], rel(pow_pos_fp64(xb, pp), pow(xb, pp)));
  }
  for (int j = 0; j < 4; ++j) atomicMax(worst + j, (unsigned long long)__double_as_longlong(e[j]));
}

}  // namespace
}  // namespace avip

using namespace avip;

extern "C" int fp64_math_check(double* max_rel_err) {
  if (!max_rel_err) return AVIP_EINVAL;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 4 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return AVIP_ENOMEM;
  }
  unsigned long long h[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemset(d, 0, sizeof(h));
  if (e == cudaSuccess) {
    fp64_math_check_kernel<<<kCheckPoints / 256, 256>>>(d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return AVIP_ECUDA;
  }
  for (int j = 0; j < 4; ++j) std::memcpy(max_rel_err + j, h + j, sizeof(double));
  return AVIP_OK;
}

extern "C" int peak_probe(int32_t which, void* stream, double* value_out) {
  if (!value_out || (which != AVIP_PROBE_FP64_FMA && which != AVIP_PROBE_HBM_COPY)) return AVIP_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return AVIP_ECUDA;
  }
  float ms = 0.f;
  if (which == AVIP_PROBE_FP64_FMA) {
    const int blocks = sms * (2048 / kProbeThreads);  // every SM full
    double* out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * kProbeThreads * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return AVIP_ENOMEM;
    }
    e = best_ms(st, [&] {
      fp64_fma_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(out, 0.9999999, 1e-7);
      return cudaGetLastError();
    }, ms);
    cudaFree(out);
    if (e == cudaSuccess && ms > 0.f)
      *value_out = 2.0 * kChains * (double)kFmaIters * blocks * kProbeThreads / (ms * 1e-3) / 1e12;  // TFLOP/s
  } else {
    void *a = nullptr, *b = nullptr;
    if (cudaMalloc(&a, kCopyBytes) != cudaSuccess || cudaMalloc(&b, kCopyBytes) != cudaSuccess) {
      cudaGetLastError();
      if (a) cudaFree(a);
      return AVIP_ENOMEM;
    }
    e = cudaMemsetAsync(a, 0, kCopyBytes, st);
    const size_t n = kCopyBytes / sizeof(int4);
    const int blocks = sms * 8;
    if (e == cudaSuccess)
      e = best_ms(st, [&] {
        copy_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(static_cast<const int4*>(a), static_cast<int4*>(b), n);
        return cudaGetLastError();
      }, ms);
    cudaFree(a);
    cudaFree(b);
    if (e == cudaSuccess && ms > 0.f) *value_out = 2.0 * (double)kCopyBytes / (ms * 1e-3) / 1e9;  // GB/s
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return AVIP_ECUDA;
  }
  return AVIP_OK;
}
