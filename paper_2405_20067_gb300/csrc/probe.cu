// probe.cu -- throughput micro-benchmarks of the two arithmetic pipes the
// evaluation kernels lean on besides the tensor cores (ndg_probe_pipe):
//   which = 0: the MUFU exponential, ex2.approx.ftz.f32 (one per
//              Gaussian-query pair in every evaluation kernel);
//   which = 1: the FP32 FMA (the plain FP32 form's pipe).
// Every thread runs 8 independent dependency chains of the instruction, so
// with a few warps per SM sub-partition the pipe, not the latency, limits the
// rate.  Each block asks for more than half of an SM's shared memory (it uses
// none), so that no SM holds two blocks: with one block per SM the clock64
// cycles a block records between two barriers around its loop are that SM's
// time, and instructions / cycles is the SM's rate per clock.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace ndg {

namespace {

template <int WHICH>
__global__ void probe_pipe_kernel(int iters, long long* __restrict__ cycles,
                                  float* __restrict__ sink) {
  float v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = 0.25f + 0.01f * (float)((threadIdx.x + j) & 15);
  const float a = 0.999f, b = 1e-3f;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (WHICH == 0)
        v[j] = ex2_approx(-v[j]);  // converges to the fixed point 2^-v = v (~0.64)
      else
        v[j] = fmaf(v[j], a, b);
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += v[j];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

constexpr int kProbeSmem = 120 * 1024;  // > half of the 228 KB of an SM: one block per SM

int launch_probe_pipe(int which, int blocks, int threads, int iters, long long* cycles,
                      float* sink, cudaStream_t s) {
  if (which == 0) {
    cudaFuncSetAttribute(probe_pipe_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kProbeSmem);
    probe_pipe_kernel<0><<<blocks, threads, kProbeSmem, s>>>(iters, cycles, sink);
  } else {
    cudaFuncSetAttribute(probe_pipe_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kProbeSmem);
    probe_pipe_kernel<1><<<blocks, threads, kProbeSmem, s>>>(iters, cycles, sink);
  }
  return 1;
}

}  // namespace ndg
