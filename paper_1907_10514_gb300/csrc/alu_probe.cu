// alu_probe.cu -- issue-rate probe of the pipes the step kernels use (sm_103a).
//
// The step kernel's roofline is an ALU roofline: FP32 lanes for the pair arithmetic,
// MUFU for rsqrt, FP64 for the epilogue.  This probe measures each pipe's throughput
// (lane operations per SM clock) with independent dependency chains in every thread,
// so the roofline is stated from measured unit counts rather than assumed ones.
#include <cuda_runtime.h>

#include <cstdint>

#include "iontrap.h"

namespace {

constexpr int kChains = 8;

__device__ __forceinline__ float probe_rsqrt(float x) {
  float r;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <int KIND>
__global__ void k_alu(long long iters, float* sink, unsigned long long* clk) {
  unsigned long long c0 = 0, t0 = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    asm volatile("mov.u64 %0, %%clock64;" : "=l"(c0));
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  }
  const float seed = 1.0f + 1e-6f * threadIdx.x;
  float acc = 0.0f;
  if (KIND == 0) {  // FFMA
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + k;
    for (long long it = 0; it < iters; ++it)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], 0.9999f, 1e-4f);
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc += a[k];
  } else if (KIND == 1 || KIND == 4) {  // FFMA2 / FADD2 (two FP32 lanes per instruction)
    float2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2(seed + k, seed - k);
    const float2 m = make_float2(0.9999f, 0.9998f), c = make_float2(1e-4f, 2e-4f);
    for (long long it = 0; it < iters; ++it)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = (KIND == 1) ? __ffma2_rn(a[k], m, c) : __fadd2_rn(a[k], c);
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc += a[k].x + a[k].y;
  } else if (KIND == 2) {  // MUFU rsqrt
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + k;
    for (long long it = 0; it < iters; ++it)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = probe_rsqrt(a[k]);
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc += a[k];
  } else if (KIND == 5) {  // FP32 <-> FP64 conversions (two per iteration)
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + k;
    for (long long it = 0; it < iters; ++it)
#pragma unroll
      for (int k = 0; k < kChains; ++k) {
        double d;
        asm volatile("cvt.f64.f32 %0, %1;" : "=d"(d) : "f"(a[k]));
        asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(a[k]) : "d"(d));
      }
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc += a[k];
  } else if (KIND == 3) {  // DFMA
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + k;
    for (long long it = 0; it < iters; ++it)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], 0.9999, 1e-4);
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc += (float)a[k];
  }
  if (acc == 123.456f) sink[threadIdx.x] = acc;  // keeps the chains live
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long c1, t1;
    asm volatile("mov.u64 %0, %%clock64;" : "=l"(c1));
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    clk[0] = c1 - c0;
    clk[1] = t1 - t0;
  }
}

}  // namespace

extern "C" int iontrap_alu_probe(int kind, long long iters, double* lane_ops_per_clk_per_sm, double* sm_mhz) {
  if (kind < 0 || kind > 5 || iters < 1 || !lane_ops_per_clk_per_sm) return IONTRAP_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IONTRAP_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 8;
  float* sink = nullptr;
  unsigned long long* clk = nullptr;
  if (cudaMalloc(&sink, threads * sizeof(float)) != cudaSuccess) return IONTRAP_ENOMEM;
  if (cudaMalloc(&clk, 2 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaFree(sink);
    return IONTRAP_ENOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&](long long n) {
    switch (kind) {
      case 0: k_alu<0><<<blocks, threads>>>(n, sink, clk); break;
      case 1: k_alu<1><<<blocks, threads>>>(n, sink, clk); break;
      case 2: k_alu<2><<<blocks, threads>>>(n, sink, clk); break;
      case 3: k_alu<3><<<blocks, threads>>>(n, sink, clk); break;
      case 5: k_alu<5><<<blocks, threads>>>(n, sink, clk); break;
      default: k_alu<4><<<blocks, threads>>>(n, sink, clk); break;
    }
  };
  launch(16);  // warm-up
  cudaEventRecord(e0);
  launch(iters);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  unsigned long long hc[2] = {0, 0};
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaMemcpy(hc, clk, sizeof(hc), cudaMemcpyDeviceToHost);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(clk);
  if (e != cudaSuccess) return IONTRAP_ECUDA;
  const double mhz = hc[1] ? (double)hc[0] / (double)hc[1] * 1e3 : 0.0;
  const double lanes_per_instr = (kind == 1 || kind == 4 || kind == 5) ? 2.0 : 1.0;
  const double ops = (double)blocks * threads * kChains * (double)iters * lanes_per_instr;
  const double clocks = (double)ms * 1e-3 * mhz * 1e6;
  *lane_ops_per_clk_per_sm = clocks > 0 ? ops / clocks / sms : 0.0;
  if (sm_mhz) *sm_mhz = mhz;
  return IONTRAP_OK;
}
