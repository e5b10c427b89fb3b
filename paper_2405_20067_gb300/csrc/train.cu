// train.cu -- Adam over the raw parameters and the Section 3.3 refinement
// (materialisation of child Gaussians) behind ndg_adam / ndg_densify.
#include "common.cuh"
#include "internal.h"
#include "kernels.h"

namespace ndg {

// ---- Adam -------------------------------------------------------------------
__global__ void __launch_bounds__(256) adam_kernel(AdamArgs a) {
  const AdamSeg sg = a.seg[blockIdx.y];
  const int t = *a.step + 1;
  const float c1 = 1.0f - powf(a.b1, (float)t);
  const float c2 = 1.0f - powf(a.b2, (float)t);
  const float step = a.lr / c1;
  const float rc2 = 1.0f / sqrtf(c2);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < sg.n;
       i += (long long)gridDim.x * blockDim.x) {
    const float g = sg.g[i];
    const float m = fmaf(a.b1, sg.m[i], (1.0f - a.b1) * g);
    const float v = fmaf(a.b2, sg.v[i], (1.0f - a.b2) * g * g);
    sg.m[i] = m;
    sg.v[i] = v;
    sg.p[i] -= step * m / (sqrtf(v) * rc2 + a.eps);
  }
}

__global__ void step_inc_kernel(int* step) { *step += 1; }

int launch_adam(const AdamArgs& a, cudaStream_t s) {
  if (a.nseg <= 0) return 0;
  long long mx = 0;
  for (int i = 0; i < a.nseg; ++i) mx = a.seg[i].n > mx ? a.seg[i].n : mx;
  unsigned bx = (unsigned)ceil_div<long long>(mx > 0 ? mx : 1, 256);
  if (bx > 4096) bx = 4096;
  adam_kernel<<<dim3(bx, a.nseg), 256, 0, s>>>(a);
  step_inc_kernel<<<1, 1, 0, s>>>(a.step);
  return 2;
}

// ---- densify ------------------------------------------------------------------
// Order-preserving map of a float to an unsigned key.
__device__ __forceinline__ uint32_t ord_key(float v) {
  uint32_t u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// One block: flags, capacity selection (the `room` brightest, ties at the
// boundary all left out: the smallest key tau with count(key >= tau) <= room),
// ranks in index order, the new row count.
__global__ void __launch_bounds__(1024) densify_select_kernel(DensifyArgs a) {
  __shared__ int red[32];
  __shared__ long long carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto block_sum = [&](int v) -> int {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    __syncthreads();
    return s;
  };
  int local = 0;
  for (int g = tid; g < a.G; g += blockDim.x) {
    int f = a.has_children && (a.c_alpha_raw[g] > a.a_thr);
    a.flag[g] = f;
    local += f;
  }
  const int nflag = block_sum(local);
  const int room = a.G_cap - a.G;
  if (nflag > room) {
    unsigned long long lo = 0, hi = 1ull << 32;
    while (lo < hi) {
      const unsigned long long mid = (lo + hi) >> 1;
      int c = 0;
      for (int g = tid; g < a.G; g += blockDim.x)
        c += a.flag[g] && (unsigned long long)ord_key(a.c_alpha_raw[g]) >= mid;
      c = block_sum(c);
      if (c <= room) hi = mid; else lo = mid + 1;
    }
    for (int g = tid; g < a.G; g += blockDim.x)
      if (a.flag[g] && (unsigned long long)ord_key(a.c_alpha_raw[g]) < lo) a.flag[g] = 0;
    __syncthreads();
  }
  // ranks in index order
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < a.G; base += blockDim.x) {
    const int g = base + tid;
    const int f = g < a.G ? a.flag[g] : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) red[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      before += w < warp ? red[w] : 0;
      total += red[w];
    }
    if (f) a.rank[g] = (int)(carry + before + __popc(bal & ((1u << lane) - 1u)));
    __syncthreads();
    if (tid == 0) carry += total;
    __syncthreads();
  }
  if (tid == 0) *a.G_new = a.G + (int)carry;
}

__device__ __forceinline__ void zero_row(float* p, long long row, int width) {
  if (!p) return;
  for (int i = 0; i < width; ++i) p[row * width + i] = 0.0f;
}

template <int N>
__global__ void __launch_bounds__(128) densify_materialize_kernel(DensifyArgs a) {
  constexpr int P = tri(N);
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.G || !a.flag[g]) return;
  const int d = a.G + a.rank[g];
  double L[P], U[P];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const double v = (double)a.theta[(size_t)g * P + tri(i) + j];
      const double u = (double)a.u_theta[(size_t)g * P + tri(i) + j];
      L[tri(i) + j] = (i == j) ? exp(v) : 2.0 / (1.0 + exp(-v)) - 1.0;
      U[tri(i) + j] = (i == j) ? exp(u) : 2.0 / (1.0 + exp(-u)) - 1.0;
    }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k <= i; ++k) s = fma(L[tri(i) + k], (double)a.m_u[(size_t)g * N + k], s);
    a.mean[(size_t)d * N + i] = (float)(s + (double)a.mean[(size_t)g * N + i]);
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      double lc = 0.0;
#pragma unroll
      for (int k = j; k <= i; ++k) lc = fma(L[tri(i) + k], U[tri(k) + j], lc);
      double th;
      if (i == j) {
        th = log(lc);
      } else {
        const double lim = 1.0 - 1e-6;
        lc = lc > lim ? lim : (lc < -lim ? -lim : lc);
        th = log((1.0 + lc) / (1.0 - lc));
      }
      a.theta[(size_t)d * P + tri(i) + j] = (float)th;
    }
  }
  a.alpha_raw[d] = a.c_alpha_raw[g];
#pragma unroll
  for (int c = 0; c < 3; ++c) a.color_raw[(size_t)d * 3 + c] = a.c_color_raw[(size_t)g * 3 + c];
  for (int mom = 0; mom < 2; ++mom) {
    const MomentPtrs& mp = a.mom[mom];
    zero_row(mp.mean, d, N);
    zero_row(mp.theta, d, P);
    zero_row(mp.alpha_raw, d, 1);
    zero_row(mp.color_raw, d, 3);
  }
  a.fresh[g] = 1;
  a.fresh[d] = 1;
}

template <int N>
__global__ void __launch_bounds__(128) densify_reinit_kernel(DensifyArgs a) {
  constexpr int P = tri(N), NR = P + N + 4;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= *a.G_new) return;
  if (a.has_children && !a.fresh[g]) return;
  const float* xi = a.noise + (size_t)g * NR;
#pragma unroll
  for (int i = 0; i < P; ++i) a.u_theta[(size_t)g * P + i] = 0.05f * xi[i];
#pragma unroll
  for (int i = 0; i < N; ++i) a.m_u[(size_t)g * N + i] = 0.1f * xi[P + i];
  a.c_alpha_raw[g] = a.a_child0 + 0.1f * xi[P + N];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    a.c_color_raw[(size_t)g * 3 + c] = a.color_raw[(size_t)g * 3 + c] + 0.1f * xi[P + N + 1 + c];
  for (int mom = 0; mom < 2; ++mom) {
    const MomentPtrs& mp = a.mom[mom];
    zero_row(mp.u_theta, g, P);
    zero_row(mp.m_u, g, N);
    zero_row(mp.c_alpha_raw, g, 1);
    zero_row(mp.c_color_raw, g, 3);
  }
}

#define NDG_CASE_N(n, call) case n: call(n); break;
#define NDG_SWITCH_N(N, call)                                                         \
  switch (N) {                                                                        \
    NDG_CASE_N(1, call) NDG_CASE_N(2, call) NDG_CASE_N(3, call) NDG_CASE_N(4, call)   \
    NDG_CASE_N(5, call) NDG_CASE_N(6, call) NDG_CASE_N(7, call) NDG_CASE_N(8, call)   \
    NDG_CASE_N(9, call) NDG_CASE_N(10, call) NDG_CASE_N(11, call) NDG_CASE_N(12, call) \
    default: break;                                                                   \
  }

int launch_densify(int N, const DensifyArgs& a, cudaStream_t s) {
  cudaMemsetAsync(a.fresh, 0, sizeof(int) * (size_t)(a.G_cap > 0 ? a.G_cap : 1), s);
  densify_select_kernel<<<1, 1024, 0, s>>>(a);
  const unsigned bg = (unsigned)ceil_div(a.G > 0 ? a.G : 1, 128);
  const unsigned bc = (unsigned)ceil_div(a.G_cap > 0 ? a.G_cap : 1, 128);
#define L_MAT(n) densify_materialize_kernel<n><<<bg, 128, 0, s>>>(a)
  NDG_SWITCH_N(N, L_MAT)
#undef L_MAT
#define L_RE(n) densify_reinit_kernel<n><<<bc, 128, 0, s>>>(a)
  NDG_SWITCH_N(N, L_RE)
#undef L_RE
  return 3;  // select, materialise, re-initialise (plus one memset)
}

}  // namespace ndg
