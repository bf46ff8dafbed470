// pipes.cu -- microbenchmarks of the arithmetic pipes the hot path uses, for
// the roofline denominators: FP64 FMA (the plain path and the certificates),
// FP32 FMA and packed f32x2 FMA (the mixed path's sweeps), and the TF32
// mma.sync.m16n8k8 rate of the tensor pipe (the scan's 3xTF32 products).
// Each thread (warp, for the mma) runs independent chains (enough to cover
// the pipe latency) over a grid of several CTAs per SM; rate = 2 flops per
// multiply-add / CUDA-event time.
#include <cuda_runtime.h>
#include <cstdint>

#include "common.cuh"

namespace rlqr {
namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void k_pipe_fma(T *out, int iters, T a, T b) {
  T acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_pipe_fma2(float *out, int iters, float a, float b) {
  float2 acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = make_float2((float)threadIdx.x, (float)c);
  const float2 a2 = bcast2(a), b2 = bcast2(b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fma2(acc[c], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c].x + acc[c].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Independent accumulator tiles per warp of the TF32 mma chain.
constexpr int kMmaChains = 8;

// Back-to-back mma.sync.m16n8k8 TF32 with FP32 accumulation (2 * 16 * 8 * 8
// flops each) on kMmaChains independent accumulators per warp.  The operands
// are small constants (their TF32 bit patterns), so the sums stay finite.
__global__ void k_pipe_tf32(float *out, int iters) {
  float acc[kMmaChains][4];
#pragma unroll
  for (int c = 0; c < kMmaChains; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[c][j] = 0.f;
  const uint32_t a = __float_as_uint(1e-3f) & 0xffffe000u, b = __float_as_uint(1e-3f) & 0xffffe000u;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kMmaChains; ++c)
      asm volatile(
          "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, "
          "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
          : "+f"(acc[c][0]), "+f"(acc[c][1]), "+f"(acc[c][2]), "+f"(acc[c][3])
          : "r"(a), "r"(a), "r"(a), "r"(a), "r"(b), "r"(b));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kMmaChains; ++c) s += acc[c][0] + acc[c][1] + acc[c][2] + acc[c][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Best of `reps` timed launches (after one warm-up) in milliseconds, or -1.
template <typename F>
float time_best(F launch, int reps) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1.f;
  }
  float best = -1.f;
  launch();
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best < 0.f || ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return (cudaGetLastError() == cudaSuccess) ? best : -1.f;
}

}  // namespace
}  // namespace rlqr

using namespace rlqr;

static int pipe_blocks() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms * 4;
}

extern "C" size_t rlqr_measure_pipes_bytes(void) {
  return (size_t)pipe_blocks() * 256 * sizeof(double);
}

extern "C" rlqr_status rlqr_measure_pipes(void *scratch, size_t scratch_bytes, double *fp64_tflops,
                                          double *fp32_tflops, double *fp32x2_tflops) {
  if (!fp64_tflops || !fp32_tflops || !fp32x2_tflops) return RLQR_ERR_ARG;
  const int threads = 256, blocks = pipe_blocks();
  if (blocks <= 0) return RLQR_ERR_CUDA;
  void *buf = scratch;
  if (!buf || scratch_bytes < (size_t)blocks * threads * sizeof(double) ||
      (reinterpret_cast<uintptr_t>(buf) % sizeof(double)) != 0)
    return RLQR_ERR_WORKSPACE;
  const double lanes = (double)blocks * threads * kChains;
  const int it64 = 2048, it32 = 32768;
  const float ms64 = time_best([&] {
    k_pipe_fma<double><<<blocks, threads>>>((double *)buf, it64, 1.0000001, 1e-9);
  }, 5);
  const float ms32 = time_best([&] {
    k_pipe_fma<float><<<blocks, threads>>>((float *)buf, it32, 1.0000001f, 1e-9f);
  }, 5);
  const float ms2 = time_best([&] {
    k_pipe_fma2<<<blocks, threads>>>((float *)buf, it32, 1.0000001f, 1e-9f);
  }, 5);
  if (ms64 <= 0.f || ms32 <= 0.f || ms2 <= 0.f) return RLQR_ERR_CUDA;
  *fp64_tflops = 2.0 * lanes * it64 / (ms64 * 1e-3) / 1e12;
  *fp32_tflops = 2.0 * lanes * it32 / (ms32 * 1e-3) / 1e12;
  *fp32x2_tflops = 2.0 * 2.0 * lanes * it32 / (ms2 * 1e-3) / 1e12;
  return RLQR_OK;
}

extern "C" rlqr_status rlqr_measure_tf32(void *scratch, size_t scratch_bytes,
                                         double *tf32_tflops) {
  if (!tf32_tflops) return RLQR_ERR_ARG;
  const int threads = 256, blocks = pipe_blocks();
  if (blocks <= 0) return RLQR_ERR_CUDA;
  if (!scratch || scratch_bytes < (size_t)blocks * threads * sizeof(float) ||
      (reinterpret_cast<uintptr_t>(scratch) % sizeof(float)) != 0)
    return RLQR_ERR_WORKSPACE;
  const int iters = 4096;
  const float ms = time_best([&] {
    k_pipe_tf32<<<blocks, threads>>>((float *)scratch, iters);
  }, 5);
  if (ms <= 0.f) return RLQR_ERR_CUDA;
  const double mmas = (double)blocks * (threads / 32) * kMmaChains * iters;
  *tf32_tflops = 2.0 * 16 * 8 * 8 * mmas / (ms * 1e-3) / 1e12;
  return RLQR_OK;
}
