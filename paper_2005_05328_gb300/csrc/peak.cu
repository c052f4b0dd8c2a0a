// peak.cu -- FP32 arithmetic peaks of the device, measured by the library's
// own micro-benchmarks: the roofline denominators of the tree walk, whose pair
// arithmetic (Sec. 2.1 short-range force) runs on the FP32 FMA pipe and the
// special-function unit (reciprocal square root, base-2 exponential).
//
// FMA: every thread runs 8 independent FMA chains (enough to cover the pipe
// latency at 8 warps per scheduler); one FFMA = 2 flop.  SFU: 4 independent
// chains of reciprocal square roots (one MUFU op each).  Each kernel is timed
// with CUDA events on its stream; the best of `reps` launches is reported.
#include <algorithm>

#include "common.cuh"

namespace dzs {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 4;

__global__ void __launch_bounds__(kPeakThreads) k_fma_chains(int iters, float b, float c, float* sink) {
  float a0 = threadIdx.x * 1e-7f, a1 = a0 + 1e-7f, a2 = a0 + 2e-7f, a3 = a0 + 3e-7f;
  float a4 = a0 + 4e-7f, a5 = a0 + 5e-7f, a6 = a0 + 6e-7f, a7 = a0 + 7e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a0 = fmaf(a0, b, c);
      a1 = fmaf(a1, b, c);
      a2 = fmaf(a2, b, c);
      a3 = fmaf(a3, b, c);
      a4 = fmaf(a4, b, c);
      a5 = fmaf(a5, b, c);
      a6 = fmaf(a6, b, c);
      a7 = fmaf(a7, b, c);
    }
  }
  const float s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  if (s == 1234.5f) sink[blockIdx.x] = s;  // keeps the chains alive; never true for these inputs
}

__global__ void __launch_bounds__(kPeakThreads) k_sfu_chains(int iters, float* sink) {
  float a0 = 1.0f + threadIdx.x * 1e-6f, a1 = a0 + 0.25f, a2 = a0 + 0.5f, a3 = a0 + 0.75f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a0 = rsqrtf(a0);
      a1 = rsqrtf(a1);
      a2 = rsqrtf(a2);
      a3 = rsqrtf(a3);
    }
  }
  const float s = (a0 + a1) + (a2 + a3);
  if (s == 1234.5f) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace dzs

extern "C" dzs_status dzs_measure_fp32_peaks(int32_t device, int32_t reps, double* fma_tflops, double* sfu_gops) {
  using namespace dzs;
  if (reps < 1 || (!fma_tflops && !sfu_gops)) return DZS_EINVAL;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return DZS_EDEVICE;
  if (cudaSetDevice(device) != cudaSuccess) return DZS_EDEVICE;
  dzs_status st = DZS_OK;
  cudaStream_t s = nullptr;
  cudaEvent_t ea = nullptr, eb = nullptr;
  float* sink = nullptr;
  const int nsm = sm_count();
  const int blocks = nsm * kPeakBlocksPerSm;
  const int fma_iters = 4096, sfu_iters = 2048;
  double best_fma = 0, best_sfu = 0;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&ea) != cudaSuccess || cudaEventCreate(&eb) != cudaSuccess ||
      cudaMalloc(&sink, sizeof(float) * blocks) != cudaSuccess) {
    st = DZS_ECUDA;
  }
  for (int r = 0; st == DZS_OK && r <= reps; ++r) {  // launch 0 warms up
    float ms = 0;
    if (fma_tflops) {
      cudaEventRecord(ea, s);
      k_fma_chains<<<blocks, kPeakThreads, 0, s>>>(fma_iters, 0.999999f, 1e-7f, sink);
      cudaEventRecord(eb, s);
      if (cudaEventSynchronize(eb) != cudaSuccess || cudaEventElapsedTime(&ms, ea, eb) != cudaSuccess) {
        st = DZS_ECUDA;
        break;
      }
      const double flop = 2.0 * 8 * 16 * (double)fma_iters * blocks * kPeakThreads;
      if (r > 0 && ms > 0) best_fma = std::max(best_fma, flop / (ms * 1e-3) / 1e12);
    }
    if (sfu_gops) {
      cudaEventRecord(ea, s);
      k_sfu_chains<<<blocks, kPeakThreads, 0, s>>>(sfu_iters, sink);
      cudaEventRecord(eb, s);
      if (cudaEventSynchronize(eb) != cudaSuccess || cudaEventElapsedTime(&ms, ea, eb) != cudaSuccess) {
        st = DZS_ECUDA;
        break;
      }
      const double ops = 4.0 * 16 * (double)sfu_iters * blocks * kPeakThreads;
      if (r > 0 && ms > 0) best_sfu = std::max(best_sfu, ops / (ms * 1e-3) / 1e9);
    }
  }
  if (st == DZS_OK && cudaGetLastError() != cudaSuccess) st = DZS_ECUDA;
  if (sink) cudaFree(sink);
  if (ea) cudaEventDestroy(ea);
  if (eb) cudaEventDestroy(eb);
  if (s) cudaStreamDestroy(s);
  cudaSetDevice(prev);
  if (st == DZS_OK) {
    if (fma_tflops) *fma_tflops = best_fma;
    if (sfu_gops) *sfu_gops = best_sfu;
  }
  return st;
}
