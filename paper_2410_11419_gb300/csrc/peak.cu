// Measured ALU peaks of the device: the denominators of the roofline of the
// ALU-bound composites (every (pixel, splat) test is FP32 fused multiply-adds,
// a compare and one MUFU ex2).  Timed micro-kernels, not an operation of the
// paper.
#include <cuda_runtime.h>

#include "gs3_internal.cuh"

namespace gs3 {
namespace {

constexpr int kChains = 8;    // independent dependency chains per thread
constexpr int kUnroll = 16;   // chain steps per loop iteration
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 8;  // 64 warps per SM

// kChains x kUnroll FMAs per iteration on values that stay bounded
// (a -> a b + c with b just below 1); the sum is stored only if it hits an
// impossible value, which the compiler cannot know.
__global__ void __launch_bounds__(kPeakThreads) k_ffma_peak(float* out, float b, float c, int iters) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 1e-3f * (float)threadIdx.x + (float)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -1.2345e30f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// kChains x kUnroll ex2 per iteration: x -> 2^(-x) (values stay in (0, 1]).
__global__ void __launch_bounds__(kPeakThreads) k_ex2_peak(float* out, int iters) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 1e-3f * (float)threadIdx.x + 0.1f * (float)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        float y;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-a[i]));
        a[i] = y;
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -1.2345e30f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace gs3

using namespace gs3;

extern "C" gs3_status gs3_measure_alu_peak(int32_t repeats, double* ffma_tflops, double* ex2_gops) {
  if (!ffma_tflops || !ex2_gops || repeats < 1 || repeats > 100) {
    set_last_error("gs3_measure_alu_peak: need two outputs and 1 <= repeats <= 100");
    return GS3_ERR_INVALID_ARG;
  }
  const int blocks = device_sm_count() * kPeakBlocksPerSm;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(float) * (size_t)blocks * kPeakThreads);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int ffma_iters = 8192, ex2_iters = 1024;
  double best_ffma = 0.0, best_ex2 = 0.0;
  for (int pass = 0; e == cudaSuccess && pass <= repeats; ++pass) {  // pass 0 warms up
    for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
      cudaEventRecord(e0);
      if (kind == 0)
        k_ffma_peak<<<blocks, kPeakThreads>>>(out, 0.9999999f, 1e-7f, ffma_iters);
      else
        k_ex2_peak<<<blocks, kPeakThreads>>>(out, ex2_iters);
      count_launch();
      cudaEventRecord(e1);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess || pass == 0 || ms <= 0.f) continue;
      const double ops = (double)blocks * kPeakThreads * kChains * kUnroll * (kind == 0 ? ffma_iters : ex2_iters);
      if (kind == 0) {
        const double tf = 2.0 * ops / (ms * 1e-3) / 1e12;
        if (tf > best_ffma) best_ffma = tf;
      } else {
        const double g = ops / (ms * 1e-3) / 1e9;
        if (g > best_ex2) best_ex2 = g;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) {
    set_last_error("gs3_measure_alu_peak: CUDA call failed");
    return GS3_ERR_CUDA;
  }
  *ffma_tflops = best_ffma;
  *ex2_gops = best_ex2;
  return GS3_OK;
}
