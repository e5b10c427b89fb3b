// eval.cu -- mixture evaluation (Eq. 1, Eq. 8), the L2 loss, and the
// analytic backward pass behind ndg_forward / ndg_loss_l2 / ndg_backward.
//
// Forward (one CTA per tile, one thread per query): the tile's candidate
// records (M = L^{-1} packed, m, w; 16-byte rows) are staged through shared
// memory in chunks and read back as broadcasts; per pair the thread forms
// d = x - m, z = M d, s = |z|^2, e = 2^(-s log2(e) / 2) and accumulates w e.
//
// Backward (one CTA per tile, one thread per candidate): the tile's queries
// and upstream gradients sit in shared memory; each thread keeps its
// Gaussian's record and its partial sums in registers and loops over the
// queries (broadcast reads), producing one partial record per candidate
// entry: sum beta z d^T (lower), sum beta z, sum dy e, beta = e sum_c dy_c w_c.
// The entries are then transposed to Gaussian-major order by a stable radix
// sort, summed per Gaussian in entry order (no atomics, bit-reproducible)
// and chained to the raw parameters (Eq. 2, 6-8) by chain_kernel.
#include "common.cuh"
#include "internal.h"
#include "kernels.h"

namespace ndg {

// ---- forward ----------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256) fwd_kernel(FwdArgs a) {
  constexpr int P = tri(N), R = rec_floats(N), R4 = R / 4;
  constexpr int CH = 64;
  __shared__ __align__(16) float srec[CH * R];
  const long long t = blockIdx.x;
  const long long q = t * a.tile + threadIdx.x;
  const bool active = threadIdx.x < a.tile && q < a.Q;
  float x[N];
#pragma unroll
  for (int d = 0; d < N; ++d) x[d] = active ? a.x[q * N + d] : 0.0f;
  const long long beg = a.offsets[t], end = a.offsets[t + 1];
  float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f;
  for (long long c0 = beg; c0 < end; c0 += CH) {
    const int n = (int)(end - c0 < CH ? end - c0 : CH);
    for (int idx = threadIdx.x; idx < n * R4; idx += blockDim.x) {
      const int row = idx / R4, col = idx - row * R4;
      const int g = a.ids[c0 + row];
      // an index outside this mixture (a stale list) reads as a zero-weight row
      reinterpret_cast<float4*>(srec)[idx] =
          (unsigned)g < (unsigned)a.Ge
              ? __ldg(reinterpret_cast<const float4*>(a.rec) + (size_t)g * R4 + col)
              : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
      const float* r = srec + j * R;
      float d[N];
#pragma unroll
      for (int i = 0; i < N; ++i) d[i] = x[i] - r[P + i];
      float s = 0.0f;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float z = 0.0f;
#pragma unroll
        for (int k = 0; k <= i; ++k) z = fmaf(r[tri(i) + k], d[k], z);
        s = fmaf(z, z, s);
      }
      const float e = ex2_approx(s * kNegHalfLog2e);
      acc0 = fmaf(r[P + N + 0], e, acc0);
      acc1 = fmaf(r[P + N + 1], e, acc1);
      acc2 = fmaf(r[P + N + 2], e, acc2);
    }
    __syncthreads();
  }
  if (active) {
    a.y[q * 3 + 0] = acc0;
    a.y[q * 3 + 1] = acc1;
    a.y[q * 3 + 2] = acc2;
  }
}

// ---- loss ---------------------------------------------------------------------
constexpr int LOSS_BLOCKS = 512;

__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ y,
                                                   const float* __restrict__ target,
                                                   float* __restrict__ dy, long long n, double scale,
                                                   double* __restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double d = (double)y[i] - (double)target[i];
    dy[i] = (float)(d * scale);
    acc += d * d;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(LOSS_BLOCKS) loss_final_kernel(const double* __restrict__ part,
                                                                 long long n, double* loss) {
  __shared__ double sh[LOSS_BLOCKS];
  sh[threadIdx.x] = part[threadIdx.x];
  __syncthreads();
  for (int s = LOSS_BLOCKS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = n > 0 ? sh[0] / (double)n : 0.0;
}

// ---- backward partials ------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256, 1) bwd_kernel(BwdArgs a) {
  constexpr int P = tri(N), R = rec_floats(N), RP = part_floats(N);
  constexpr int QS = (N + 3 + 3) / 4 * 4;  // x (N) and dy (3) per query, 16-byte rows
  __shared__ __align__(16) float sq[NDG_MAX_TILE * QS];
  const long long t = blockIdx.x;
  const long long q0 = t * a.tile;
  const int nq = (int)(a.Q - q0 < a.tile ? a.Q - q0 : a.tile);
  for (int i = threadIdx.x; i < nq * QS; i += blockDim.x) {
    const int qi = i / QS, c = i - qi * QS;
    float v = 0.0f;
    if (c < N) v = a.x[(q0 + qi) * N + c];
    else if (c < N + 3) v = a.dy[(q0 + qi) * 3 + (c - N)];
    sq[i] = v;
  }
  __syncthreads();
  const long long beg = a.offsets[t], end = a.offsets[t + 1];
  for (long long c0 = beg; c0 < end; c0 += blockDim.x) {
    const long long c = c0 + threadIdx.x;
    const bool act = c < end;
    float M[P], m[N], w[3];
    const int gid = act ? a.ids[c] : -1;
    if (act && (unsigned)gid < (unsigned)a.Ge) {
      const float* r = a.rec + (size_t)gid * R;
#pragma unroll
      for (int i = 0; i < P; ++i) M[i] = r[i];
#pragma unroll
      for (int i = 0; i < N; ++i) m[i] = r[P + i];
#pragma unroll
      for (int i = 0; i < 3; ++i) w[i] = r[P + N + i];
    } else {
#pragma unroll
      for (int i = 0; i < P; ++i) M[i] = 0.0f;
#pragma unroll
      for (int i = 0; i < N; ++i) m[i] = 0.0f;
#pragma unroll
      for (int i = 0; i < 3; ++i) w[i] = 0.0f;
    }
    float GM[P], Gz[N], Gw[3];
#pragma unroll
    for (int i = 0; i < P; ++i) GM[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < N; ++i) Gz[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) Gw[i] = 0.0f;
    for (int qi = 0; qi < nq; ++qi) {
      const float* qq = sq + qi * QS;
      float d[N], z[N];
#pragma unroll
      for (int i = 0; i < N; ++i) d[i] = qq[i] - m[i];
      float s = 0.0f;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float zi = 0.0f;
#pragma unroll
        for (int k = 0; k <= i; ++k) zi = fmaf(M[tri(i) + k], d[k], zi);
        z[i] = zi;
        s = fmaf(zi, zi, s);
      }
      const float e = ex2_approx(s * kNegHalfLog2e);
      const float g0 = qq[N], g1 = qq[N + 1], g2 = qq[N + 2];
      Gw[0] = fmaf(g0, e, Gw[0]);
      Gw[1] = fmaf(g1, e, Gw[1]);
      Gw[2] = fmaf(g2, e, Gw[2]);
      const float beta = e * fmaf(g0, w[0], fmaf(g1, w[1], g2 * w[2]));
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float bz = beta * z[i];
        Gz[i] += bz;
#pragma unroll
        for (int k = 0; k <= i; ++k) GM[tri(i) + k] = fmaf(bz, d[k], GM[tri(i) + k]);
      }
    }
    if (act) {
      float* out = a.part + (size_t)c * RP;
      float buf[RP];
#pragma unroll
      for (int i = 0; i < P; ++i) buf[i] = GM[i];
#pragma unroll
      for (int i = 0; i < N; ++i) buf[P + i] = Gz[i];
#pragma unroll
      for (int i = 0; i < 3; ++i) buf[P + N + i] = Gw[i];
#pragma unroll
      for (int i = P + N + 3; i < RP; ++i) buf[i] = 0.0f;
#pragma unroll
      for (int i = 0; i < RP; i += 4)
        *reinterpret_cast<float4*>(out + i) = make_float4(buf[i], buf[i + 1], buf[i + 2], buf[i + 3]);
    }
  }
}

// ---- per-Gaussian sums of the partial records (Gaussian-major, fixed order) --
__global__ void __launch_bounds__(256) segsum_kernel(const float* __restrict__ part, int RP,
                                                     const int32_t* __restrict__ gidx,
                                                     const long long* __restrict__ goff, int Ge,
                                                     float* __restrict__ gsum) {
  const long long e = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= Ge) return;
  const long long b = goff[e], en = goff[e + 1];
  for (int c = lane; c < RP; c += 32) {
    float acc = 0.0f;
    for (long long j = b; j < en; ++j) acc += part[(size_t)gidx[j] * RP + c];
    gsum[(size_t)e * RP + c] = acc;
  }
}

// ---- chain rule to the raw parameters --------------------------------------------
template <int N>
__device__ __forceinline__ void act_lower32(const float* __restrict__ th, float* L) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const float v = th[tri(i) + j];
      L[tri(i) + j] = (i == j) ? expf(v) : 2.0f / (1.0f + expf(-v)) - 1.0f;
    }
}

template <int N>
__device__ __forceinline__ void inv_lower(const float* L, float* M) {
#pragma unroll
  for (int j = 0; j < N; ++j) {
    M[tri(j) + j] = 1.0f / L[tri(j) + j];
#pragma unroll
    for (int i = j + 1; i < N; ++i) {
      float s = 0.0f;
#pragma unroll
      for (int k = j; k < i; ++k) s = fmaf(L[tri(i) + k], M[tri(k) + j], s);
      M[tri(i) + j] = -s / L[tri(i) + i];
    }
  }
}

// dl/dL (lower) = M^T A M^T where A = sum beta z d^T = -(dl/dM); and
// dl/dm = M^T sum beta z.
template <int N>
__device__ __forceinline__ void grad_L_m(const float* M, const float* A, const float* Gz,
                                         float* GL, float* Gm) {
  float H[N][N];  // H = A M^T, H[a][j] = sum_{b <= min(a, j)} A[a][b] M[j][b]
#pragma unroll
  for (int aa = 0; aa < N; ++aa)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float s = 0.0f;
#pragma unroll
      for (int b = 0; b <= (aa < j ? aa : j); ++b) s = fmaf(A[tri(aa) + b], M[tri(j) + b], s);
      H[aa][j] = s;
    }
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      float s = 0.0f;
#pragma unroll
      for (int aa = i; aa < N; ++aa) s = fmaf(M[tri(aa) + i], H[aa][j], s);
      GL[tri(i) + j] = s;
    }
    float g = 0.0f;
#pragma unroll
    for (int aa = i; aa < N; ++aa) g = fmaf(M[tri(aa) + i], Gz[aa], g);
    Gm[i] = g;
  }
}

template <int N>
__device__ __forceinline__ void raw_theta_grad(const float* GL, const float* L, float* out) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const float l = L[tri(i) + j];
      // d exp(t)/dt = L_ii;  d(2 sigmoid(t) - 1)/dt = (1 - L^2) / 2
      out[tri(i) + j] = GL[tri(i) + j] * (i == j ? l : 0.5f * (1.0f - l * l));
    }
}

__device__ __forceinline__ void raw_weight_grad(const float* Gw, float araw, const float* gam,
                                                float* ga, float* gg) {
  const float alpha = expf(araw);
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float cc = 1.0f / (1.0f + expf(-gam[c]));
    s = fmaf(Gw[c], alpha * cc, s);           // d w_c / d a = w_c
    gg[c] = Gw[c] * alpha * cc * (1.0f - cc);  // d w_c / d gamma_c
  }
  *ga = s;
}

template <int N>
__global__ void __launch_bounds__(128) chain_kernel(ChainArgs a) {
  constexpr int P = tri(N), RP = part_floats(N);
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.G) return;
  float L[P], M[P], GL[P], Gm[N];
  act_lower32<N>(a.theta + (size_t)g * P, L);
  inv_lower<N>(L, M);
  const float* sp = a.gsum + (size_t)g * RP;
  grad_L_m<N>(M, sp, sp + P, GL, Gm);
  if (a.has_children) {
    const float* sc = a.gsum + (size_t)(a.G + g) * RP;
    float U[P], Lc[P], Mc[P], GLc[P], Gmc[N], mu[N];
    act_lower32<N>(a.u_theta + (size_t)g * P, U);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      mu[i] = a.m_u[(size_t)g * N + i];
#pragma unroll
      for (int j = 0; j <= i; ++j) {
        float s = 0.0f;
#pragma unroll
        for (int k = j; k <= i; ++k) s = fmaf(L[tri(i) + k], U[tri(k) + j], s);
        Lc[tri(i) + j] = s;
      }
    }
    inv_lower<N>(Lc, Mc);
    grad_L_m<N>(Mc, sc, sc + P, GLc, Gmc);
    // L_c = L_p U, m_c = L_p m_u + m_p (Eq. 6-7):
    //   dl/dL_p += lower(GLc U^T) + lower(Gmc m_u^T), dl/dm_p += Gmc,
    //   dl/dU = lower(L_p^T GLc), dl/dm_u = L_p^T Gmc.
    float GU[P], gmu[N];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) {
        float s = Gmc[i] * mu[j];
#pragma unroll
        for (int k = 0; k <= j; ++k) s = fmaf(GLc[tri(i) + k], U[tri(j) + k], s);
        GL[tri(i) + j] += s;
      }
#pragma unroll
    for (int kk = 0; kk < N; ++kk) {
#pragma unroll
      for (int j = 0; j <= kk; ++j) {
        float s = 0.0f;
#pragma unroll
        for (int i = kk; i < N; ++i) s = fmaf(L[tri(i) + kk], GLc[tri(i) + j], s);
        GU[tri(kk) + j] = s;
      }
      float s = 0.0f;
#pragma unroll
      for (int i = kk; i < N; ++i) s = fmaf(L[tri(i) + kk], Gmc[i], s);
      gmu[kk] = s;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) Gm[i] += Gmc[i];
    float gu[P];
    raw_theta_grad<N>(GU, U, gu);
#pragma unroll
    for (int i = 0; i < P; ++i) a.g_u_theta[(size_t)g * P + i] = gu[i];
#pragma unroll
    for (int i = 0; i < N; ++i) a.g_m_u[(size_t)g * N + i] = gmu[i];
    float gam[3] = {a.c_color_raw[(size_t)g * 3], a.c_color_raw[(size_t)g * 3 + 1],
                    a.c_color_raw[(size_t)g * 3 + 2]};
    float ga, gg[3];
    raw_weight_grad(sc + P + N, a.c_alpha_raw[g], gam, &ga, gg);
    a.g_c_alpha[g] = ga;
#pragma unroll
    for (int c = 0; c < 3; ++c) a.g_c_color[(size_t)g * 3 + c] = gg[c];
  }
  float gt[P];
  raw_theta_grad<N>(GL, L, gt);
#pragma unroll
  for (int i = 0; i < P; ++i) a.g_theta[(size_t)g * P + i] = gt[i];
#pragma unroll
  for (int i = 0; i < N; ++i) a.g_mean[(size_t)g * N + i] = Gm[i];
  float gam[3] = {a.color_raw[(size_t)g * 3], a.color_raw[(size_t)g * 3 + 1],
                  a.color_raw[(size_t)g * 3 + 2]};
  float ga, gg[3];
  raw_weight_grad(sp + P + N, a.alpha_raw[g], gam, &ga, gg);
  a.g_alpha[g] = ga;
#pragma unroll
  for (int c = 0; c < 3; ++c) a.g_color[(size_t)g * 3 + c] = gg[c];
}

// ---- launchers -------------------------------------------------------------------
#define NDG_CASE_N(n, call) case n: call(n); break;
#define NDG_SWITCH_N(N, call)                                                         \
  switch (N) {                                                                        \
    NDG_CASE_N(1, call) NDG_CASE_N(2, call) NDG_CASE_N(3, call) NDG_CASE_N(4, call)   \
    NDG_CASE_N(5, call) NDG_CASE_N(6, call) NDG_CASE_N(7, call) NDG_CASE_N(8, call)   \
    NDG_CASE_N(9, call) NDG_CASE_N(10, call) NDG_CASE_N(11, call) NDG_CASE_N(12, call) \
    default: break;                                                                   \
  }

int launch_fwd(int N, const FwdArgs& a, long long T, cudaStream_t s) {
  if (T <= 0) return 0;
#define L_FWD(n) fwd_kernel<n><<<(unsigned)T, 256, 0, s>>>(a)
  NDG_SWITCH_N(N, L_FWD)
#undef L_FWD
  return 1;
}

int launch_loss(const float* y, const float* target, float* dy, long long n, double* part,
                double* loss, cudaStream_t s) {
  const double scale = n > 0 ? 2.0 / (double)n : 0.0;
  loss_kernel<<<LOSS_BLOCKS, 256, 0, s>>>(y, target, dy, n, scale, part);
  loss_final_kernel<<<1, LOSS_BLOCKS, 0, s>>>(part, n, loss);
  return 2;
}

int launch_bwd(int N, const BwdArgs& a, long long T, cudaStream_t s) {
  if (T <= 0) return 0;
#define L_BWD(n) bwd_kernel<n><<<(unsigned)T, 256, 0, s>>>(a)
  NDG_SWITCH_N(N, L_BWD)
#undef L_BWD
  return 1;
}

int launch_segsum(const float* part, int RP, const int32_t* gidx, const long long* goff, int Ge,
                  float* gsum, cudaStream_t s) {
  if (Ge <= 0) return 0;
  segsum_kernel<<<(unsigned)ceil_div<long long>((long long)Ge * 32, 256), 256, 0, s>>>(
      part, RP, gidx, goff, Ge, gsum);
  return 1;
}

int launch_chain(int N, const ChainArgs& a, cudaStream_t s) {
  if (a.G <= 0) return 0;
  unsigned blocks = (unsigned)ceil_div(a.G, 128);
#define L_CH(n) chain_kernel<n><<<blocks, 128, 0, s>>>(a)
  NDG_SWITCH_N(N, L_CH)
#undef L_CH
  return 1;
}

}  // namespace ndg
