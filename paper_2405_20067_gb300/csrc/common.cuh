// common.cuh -- device helpers shared by the libndg kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ndg.h"

namespace ndg {

__host__ __device__ constexpr int tri(int n) { return n * (n + 1) / 2; }
// Prepared record per evaluated Gaussian: M = L^{-1} packed lower (P), m (N),
// w (3), padded to a multiple of 4 floats (16-byte rows).
__host__ __device__ constexpr int rec_floats(int n) { return (tri(n) + n + 3 + 3) / 4 * 4; }
// Backward partial record: sum beta z d^T (P), sum beta z (N), sum dy e (3).
__host__ __device__ constexpr int part_floats(int n) { return (tri(n) + n + 3 + 3) / 4 * 4; }
__host__ __device__ constexpr int key_pad(int k) { return k <= 0 ? 0 : (k + 7) / 8 * 8; }

// Workspace header (first 256 bytes): status word and small counters.
struct WsHeader {
  int status;
  int pad0;
  long long live;  // live Gaussians after the cull prep
  int pad[60];
};

__device__ __forceinline__ void set_status(int* status, int code) {
  atomicCAS(status, 0, code);
}

// exp(x) for x <= 0 through the ex2 instruction: 2^(x log2 e).
__device__ __forceinline__ float ex2_approx(float v) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
constexpr float kNegHalfLog2e = -0.72134752044448170368f;  // -log2(e) / 2

// ---- FP32 bucket contract (Section 3.2 culling made reproducible) --------
// bucket(v) = floor((v - lo) * inv_h) with both operations rounded, NaN -> 0,
// saturated to [-2, B+1].
__device__ __forceinline__ int bucket_raw(float v, float lo, float inv_h, int B) {
  float t = __fmul_rn(__fsub_rn(v, lo), inv_h);
  if (t != t) return 0;
  if (t < -1.0f) return -2;
  if (t >= (float)(B + 1)) return B + 1;
  return (int)floorf(t);
}

__device__ __forceinline__ int clampi(int v, int a, int b) { return v < a ? a : (v > b ? b : v); }

template <typename T>
__host__ __device__ inline T ceil_div(T a, T b) { return (a + b - 1) / b; }

}  // namespace ndg
