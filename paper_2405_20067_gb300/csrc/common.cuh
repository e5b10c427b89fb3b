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
// Record of the tensor-core backward: the head as above with A = M^T M in
// place of M, followed by M itself (padded to a multiple of 4 floats).
__host__ __device__ constexpr int rec_tc_floats(int n) { return rec_floats(n) + (tri(n) + 3) / 4 * 4; }
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

// ---- tile centre ---------------------------------------------------------------
// Midpoint of the tile's bounding box (per dimension), computed by the CTA:
// the kernels evaluate z = M (x - c) - M (m - c), which keeps the products
// M x small (x - c is bounded by the tile) while giving the same z.
template <int N>
__device__ __forceinline__ void tile_centre(const float (&xa)[N], bool va, const float (&xb)[N],
                                            bool vb, float* __restrict__ sred,
                                            float* __restrict__ sctr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int d = 0; d < N; ++d) {
    float lo = INFINITY, hi = -INFINITY;
    if (va) { lo = xa[d]; hi = xa[d]; }
    if (vb) { lo = fminf(lo, xb[d]); hi = fmaxf(hi, xb[d]); }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      sred[(warp * N + d) * 2] = lo;
      sred[(warp * N + d) * 2 + 1] = hi;
    }
  }
  __syncthreads();
  if (threadIdx.x < N) {
    float lo = INFINITY, hi = -INFINITY;
    for (int w = 0; w < nw; ++w) {
      lo = fminf(lo, sred[(w * N + threadIdx.x) * 2]);
      hi = fmaxf(hi, sred[(w * N + threadIdx.x) * 2 + 1]);
    }
    sctr[threadIdx.x] = (lo <= hi) ? 0.5f * (lo + hi) : 0.0f;
  }
  __syncthreads();
}

}  // namespace ndg
