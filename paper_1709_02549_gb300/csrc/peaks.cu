// Microbenchmarks of the two on-chip peaks the image kernels are bound by:
// the FP32 FMA pipe (independent chains of paired FMAs, __ffma2_rn, the
// instruction the literal pair products use) and the shared-memory load pipe
// (conflict-free 32-bit loads, one 128-byte wavefront per warp instruction,
// the access the DAS and identity-DMAS windows use). Measurement aids for the
// roofline fractions; the paper has no counterpart.
#include <cuda_runtime.h>

#include "ptx.cuh"
#include "uwb_internal.cuh"

namespace uwb {
namespace {

constexpr int kChains = 8;       // independent float2 accumulators per thread
constexpr int kLdsUnroll = 16;   // independent shared loads per iteration

__global__ void __launch_bounds__(256) k_peak_fma(float* out, int iters, float a, float b) {
  float2 acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c)
    acc[c] = make_float2(threadIdx.x * 1e-3f + c, static_cast<float>(c) * 0.5f);
  const float2 aa = make_float2(a, a), bb = make_float2(b, b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = __ffma2_rn(acc[c], aa, bb);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c].x + acc[c].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(256) k_peak_lds(float* out, int iters) {
  __shared__ float buf[kLdsUnroll * 256];
  for (int i = threadIdx.x; i < kLdsUnroll * 256; i += blockDim.x) buf[i] = i * 1e-3f;
  __syncthreads();
  float acc[kLdsUnroll];
#pragma unroll
  for (int u = 0; u < kLdsUnroll; ++u) acc[u] = 0.f;
  // lane l of every warp reads word (base + l): consecutive words, no
  // conflicts. The loads are volatile in PTX (ld.volatile.shared) so that the
  // assembler neither merges nor hoists any of them out of the loop (the
  // words do not change).
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t sbase = static_cast<uint32_t>(__cvta_generic_to_shared(buf));
  uint32_t off = 4u * static_cast<uint32_t>(warp * 32 + lane);  // < 1024
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kLdsUnroll; ++u) {
      float v;
      asm volatile("ld.volatile.shared.f32 %0, [%1];" : "=f"(v) : "r"(sbase + off + u * 1024u));
      acc[u] += v;
    }
    off ^= 128u;  // alternate between two 32-word blocks; off stays below 1024
  }
  float s = 0.f;
#pragma unroll
  for (int u = 0; u < kLdsUnroll; ++u) s += acc[u];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Failure-detection self-check: one warp waits on a shared-memory mbarrier
// that nothing ever completes (arrival count 1, no arrival), probing it with
// the same bounded try-wait loop as the image kernels' staging wait, at most
// `probes` times. When the probes run out it records UWB_ERR_TIMEOUT in the
// status word and returns, as the staging wait does.
__global__ void __launch_bounds__(32) k_wait_selftest(int* status, long probes) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t ok = 0;
  for (long it = 0; it < probes && !ok; ++it) ok = mbar_try_wait(&bar, 0);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(status, UWB_ERR_TIMEOUT);
}

float time_ms(cudaEvent_t e0, cudaEvent_t e1) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms;
}

}  // namespace

// FP32 TFLOP/s (2 per FMA) and shared-load wavefronts per second, measured on
// the current device with 8 resident 256-thread CTAs per SM.
cudaError_t measure_peaks(int sms, double* tflops, double* wavefronts_per_s) {
  float* out = nullptr;
  const int blocks = sms * 8;
  cudaError_t e = cudaMalloc(&out, sizeof(float) * 256 * blocks);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int fma_iters = 20000, lds_iters = 4000;
  k_peak_fma<<<blocks, 256>>>(out, 100, 0.999f, 1e-3f);  // warm-up
  cudaEventRecord(e0);
  k_peak_fma<<<blocks, 256>>>(out, fma_iters, 0.999f, 1e-3f);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  const double fma_ms = time_ms(e0, e1);
  k_peak_lds<<<blocks, 256>>>(out, 10);
  cudaEventRecord(e0);
  k_peak_lds<<<blocks, 256>>>(out, lds_iters);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  const double lds_ms = time_ms(e0, e1);
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return e;
  const double fmas = static_cast<double>(blocks) * 256 * fma_iters * kChains * 2;
  *tflops = 2.0 * fmas / (fma_ms * 1e-3) / 1e12;
  const double wavefronts = static_cast<double>(blocks) * (256 / 32) * lds_iters * kLdsUnroll;
  *wavefronts_per_s = wavefronts / (lds_ms * 1e-3);
  return cudaSuccess;
}

// Runs k_wait_selftest on the current device and waits for it.
cudaError_t wait_selftest(int* status, long probes) {
  k_wait_selftest<<<1, 32>>>(status, probes);
  const cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? e : cudaDeviceSynchronize();
}

}  // namespace uwb
