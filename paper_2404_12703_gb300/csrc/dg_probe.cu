// dg_probe.cu -- arithmetic peak probes for the roofline denominators of the
// benchmark: the FP64 FMA rate (the bound of the FP64 path), the FP64 tensor
// (DMMA, mma.sync m8n8k4) rate, both issued together from the same warps (to
// tell whether the two share one pipe), and the FP32 FMA rate.
//
// Each probe is one launch of independent dependency chains per thread (eight
// per thread, so that the pipe, not the chain latency, is the limit) over a
// grid of eight 256-thread blocks per SM, timed with CUDA events after one
// warm-up launch.  Registers only: the single global store per thread keeps
// the compiler from removing the chains.
#include <cuda_runtime.h>

#include "dg_launch.h"

namespace dg {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

__device__ __forceinline__ void dmma_m8n8k4(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

// KIND 0: FP64 FMA; 1: FP64 MMA; 2: both per iteration; 3: FP32 FMA
template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS) k_peak(int iters, double seed, double* out) {
  const int tid = blockIdx.x * PROBE_THREADS + threadIdx.x;
  double acc = 0.0;
  if constexpr (KIND == 3) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = (float)seed + 1e-6f * (float)(threadIdx.x + i);
    const float m = 0.9999999f, c = 1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = fmaf(x[i], m, c);
    }
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) acc += (double)x[i];
  } else {
    double x[PROBE_CHAINS], d0[4], d1[4];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = seed + 1e-9 * (double)(threadIdx.x + i);
#pragma unroll
    for (int i = 0; i < 4; ++i) d0[i] = d1[i] = 1e-3 * (double)i;
    const double m = 0.9999999999, c = 1e-12, av = 1e-3 + 1e-12 * threadIdx.x, bv = 2e-3;
    for (int it = 0; it < iters; ++it) {
      if constexpr (KIND == 0 || KIND == 2) {
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = fma(x[i], m, c);
      }
      if constexpr (KIND == 1 || KIND == 2) {
#pragma unroll
        for (int i = 0; i < 4; ++i) dmma_m8n8k4(d0[i], d1[i], av, bv);
      }
    }
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) acc += x[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc += d0[i] + d1[i];
  }
  out[tid] = acc;
}

}  // namespace dg

using namespace dg;

extern "C" int dg_peak_probe(int kind, int iters, double* flops_per_s, double* ms, void* stream) {
  if (kind < 0 || kind > 3 || iters < 1 || !flops_per_s)
    return set_error(DG_ERR_ARG, "dg_peak_probe: kind in 0..3, iters >= 1, flops_per_s not NULL");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_error(DG_ERR_CUDA, std::string("dg_peak_probe: ") + cudaGetErrorString(e));
  const int blocks = sms * 8;
  const int64_t threads = (int64_t)blocks * PROBE_THREADS;
  cudaStream_t st = (cudaStream_t)stream;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&out, sizeof(double) * threads);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float t = 0.0f;
  if (e == cudaSuccess) {
    auto launch = [&]() {
      switch (kind) {
        case 0: k_peak<0><<<blocks, PROBE_THREADS, 0, st>>>(iters, 1.0, out); break;
        case 1: k_peak<1><<<blocks, PROBE_THREADS, 0, st>>>(iters, 1.0, out); break;
        case 2: k_peak<2><<<blocks, PROBE_THREADS, 0, st>>>(iters, 1.0, out); break;
        default: k_peak<3><<<blocks, PROBE_THREADS, 0, st>>>(iters, 1.0, out); break;
      }
      count_launch();
    };
    launch();  // warm-up
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return set_error(DG_ERR_CUDA, std::string("dg_peak_probe: ") + cudaGetErrorString(e));
  // flops: an FMA counts 2; one m8n8k4 MMA is 2 * 8 * 8 * 4 flops per warp
  const double fma_flops = 2.0 * PROBE_CHAINS * (double)iters * (double)threads;
  const double mma_flops = 512.0 * 4.0 * (double)iters * (double)(threads / 32);
  const double flops = kind == 0 || kind == 3 ? fma_flops : (kind == 1 ? mma_flops : fma_flops + mma_flops);
  *flops_per_s = flops / (t * 1e-3);
  if (ms) *ms = t;
  return DG_OK;
}
