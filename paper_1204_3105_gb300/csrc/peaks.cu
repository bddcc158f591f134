// peaks.cu - fmm2d_measure_alu_peaks: measured throughput of the units the
// FMM kernels are bound by (FP32 FMA, the MUFU log2 unit, FP64 FMA), used as
// roofline denominators.  Each kernel runs independent dependency chains in
// every thread of a full grid and is timed with CUDA events.
#include "plan.h"

namespace fmm2d {
namespace {

constexpr int PK_TH = 256, PK_ITERS = 4096;

__global__ void __launch_bounds__(PK_TH) k_peak_ffma(float *out, float b, float c) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3f + i;
  for (int it = 0; it < PK_ITERS; ++it)
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], b, c);
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == 12345.678f) out[threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_TH) k_peak_lg2(float *out, float c) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = 1.5f + threadIdx.x * 1e-4f + i * 1e-2f;
  for (int it = 0; it < PK_ITERS; ++it)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float y;
      asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[i]));
      x[i] = y + c;   // stays in (1, 4) for c = 1.25
    }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == 12345.678f) out[threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_TH) k_peak_dfma(double *out, double b, double c) {
  double x[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) x[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < PK_ITERS / 8; ++it)
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = fma(x[i], b, c);
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) s += x[i];
  if (s == 12345.678) out[threadIdx.x] = s;
}

}  // namespace
}  // namespace fmm2d

using namespace fmm2d;

extern "C" fmm2d_status fmm2d_measure_alu_peaks(double *out) {
  if (!out) return FMM2D_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FMM2D_ECUDA;
  double *buf = nullptr;
  if (cudaMalloc(&buf, PK_TH * sizeof(double)) != cudaSuccess) return FMM2D_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8;
  const double threads = (double)blocks * PK_TH;
  auto time = [&](auto launch) {
    launch();   // warm-up
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(e0);
      launch();
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = ms < best ? ms : best;
    }
    return (double)best * 1e-3;
  };
  const double t_fma = time([&] { k_peak_ffma<<<blocks, PK_TH>>>((float *)buf, 0.999f, 1e-3f); });
  const double t_lg2 = time([&] { k_peak_lg2<<<blocks, PK_TH>>>((float *)buf, 1.25f); });
  const double t_dfma = time([&] { k_peak_dfma<<<blocks, PK_TH>>>(buf, 0.999, 1e-3); });
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (err != cudaSuccess) return FMM2D_ECUDA;
  out[0] = threads * PK_ITERS * 8 * 2.0 / t_fma * 1e-12;        // FP32 TFLOP/s
  out[1] = threads * PK_ITERS * 8 / t_lg2 * 1e-9;               // lg2 Gop/s
  out[2] = threads * (PK_ITERS / 8) * 4 * 2.0 / t_dfma * 1e-12; // FP64 TFLOP/s
  out[3] = (double)sms;
  double tf32 = 0.0;
  const cudaError_t te = tc_measure_tf32(&tf32);   // tcgen05 kind::tf32, FP32 accumulate
  if (te != cudaSuccess) return FMM2D_ECUDA;
  out[4] = tf32;
  return FMM2D_OK;
}
