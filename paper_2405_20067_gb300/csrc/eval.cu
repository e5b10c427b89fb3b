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
// entry: dl/dM = -sum beta z d^T (lower), dl/dm = M^T sum beta z,
// dl/dw = sum dy e, with beta = e sum_c dy_c w_c.
// The entries are then transposed to Gaussian-major order by a stable radix
// sort, summed per Gaussian in entry order (no atomics, bit-reproducible)
// and chained to the raw parameters (Eq. 2, 6-8) by chain_kernel.
#include "common.cuh"
#include "internal.h"
#include "kernels.h"

namespace ndg {

// z' = kappa z with kappa = sqrt(log2(e) / 2): then exp(-|z|^2 / 2) = 2^(-|z'|^2).
constexpr float kKappa = 0.84932180028801904272f;
constexpr float kInvKappa = 1.17741002251547469101f;

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 ex2_f2(float2 v) { return make_float2(ex2_approx(v.x), ex2_approx(v.y)); }

// ---- forward ----------------------------------------------------------------
// One CTA of 128 threads per tile, two queries per thread; candidates are
// processed two at a time as the two lanes of packed FP32x2 instructions,
// their records interleaved in shared memory: (kappa M, -kappa M (m - c), w).
template <int N>
__global__ void __launch_bounds__(128) fwd_kernel(FwdArgs a) {
  constexpr int P = tri(N), R = rec_floats(N), R4 = R / 4;
  constexpr int RR = (2 * (P + N + 3) + 3) / 4 * 4;  // floats per candidate pair
  constexpr int CH = 64;                              // candidates per stage
  __shared__ __align__(16) float spair[CH / 2 * RR];
  __shared__ float sred[4 * N * 2];
  __shared__ float sctr[N];
  // tile of this CTA (a tile list selects a subset; surplus CTAs leave at once)
  if (a.tiles && (int)blockIdx.x >= *a.n_tiles) return;
  const long long t = a.tiles ? (long long)a.tiles[blockIdx.x] : (long long)blockIdx.x;
  const int tid = threadIdx.x;
  const long long q0 = t * a.tile;
  const int nq = (int)(a.Q - q0 < a.tile ? a.Q - q0 : a.tile);
  const bool va = tid < nq, vb = tid + 128 < nq;
  float xa[N], xb[N];
#pragma unroll
  for (int d = 0; d < N; ++d) {
    xa[d] = va ? a.x[(q0 + tid) * N + d] : 0.0f;
    xb[d] = vb ? a.x[(q0 + tid + 128) * N + d] : 0.0f;
  }
  tile_centre<N>(xa, va, xb, vb, sred, sctr);
  float2 xa2[N], xb2[N];
#pragma unroll
  for (int d = 0; d < N; ++d) {
    xa2[d] = f2(xa[d] - sctr[d]);
    xb2[d] = f2(xb[d] - sctr[d]);
  }
  float2 acca[3] = {f2(0.f), f2(0.f), f2(0.f)}, accb[3] = {f2(0.f), f2(0.f), f2(0.f)};
  const long long beg = a.offsets[t], end = a.offsets[t + 1];
  for (long long c0 = beg; c0 < end; c0 += CH) {
    const int n = (int)(end - c0 < CH ? end - c0 : CH);
    if (tid < CH) {
      // stage candidate tid: scaled M, -kappa M (m - c), w (zeros past the end)
      float M[P], m[N], w[3];
      const int g = tid < n ? a.ids[c0 + tid] : -1;
      if ((unsigned)g < (unsigned)a.Ge) {
        // record [M, m, w] (M first), or a record whose M sits at mat_off4
        const int stride4 = a.rec_stride4 > 0 ? a.rec_stride4 : R4;
        const float4* src = reinterpret_cast<const float4*>(a.rec) + (size_t)g * stride4;
        float buf[R];
#pragma unroll
        for (int i = 0; i < R4; ++i) {
          float4 v = __ldg(src + i);
          buf[4 * i] = v.x; buf[4 * i + 1] = v.y; buf[4 * i + 2] = v.z; buf[4 * i + 3] = v.w;
        }
        if (a.mat_off4 > 0) {
          const float* ms = reinterpret_cast<const float*>(src + a.mat_off4);
#pragma unroll
          for (int i = 0; i < P; ++i) buf[i] = __ldg(ms + i);
        }
#pragma unroll
        for (int i = 0; i < P; ++i) M[i] = kKappa * buf[i];
#pragma unroll
        for (int i = 0; i < N; ++i) m[i] = buf[P + i] - sctr[i];
#pragma unroll
        for (int i = 0; i < 3; ++i) w[i] = buf[P + N + i];
      } else {
#pragma unroll
        for (int i = 0; i < P; ++i) M[i] = 0.0f;
#pragma unroll
        for (int i = 0; i < N; ++i) m[i] = 0.0f;
#pragma unroll
        for (int i = 0; i < 3; ++i) w[i] = 0.0f;
      }
      float* dst = spair + (tid >> 1) * RR + (tid & 1);
#pragma unroll
      for (int i = 0; i < P; ++i) dst[2 * i] = M[i];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float bi = 0.0f;
#pragma unroll
        for (int k = 0; k <= i; ++k) bi = fmaf(M[tri(i) + k], m[k], bi);
        dst[2 * (P + i)] = -bi;
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) dst[2 * (P + N + i)] = w[i];
    }
    __syncthreads();
    // two-level summation: the stage's contributions are summed on their own
    // and the stage sum is added to the running total, so that the rounding
    // error grows with the stage length plus the number of stages, not with
    // the tile's whole candidate count (tens of thousands at the benchmark's
    // density)
    float2 pa[3] = {f2(0.f), f2(0.f), f2(0.f)}, pb[3] = {f2(0.f), f2(0.f), f2(0.f)};
    const int npairs = (n + 1) >> 1;
    for (int p = 0; p < npairs; ++p) {
      const float2* r = reinterpret_cast<const float2*>(spair + p * RR);
      float2 sa = f2(0.f), sb = f2(0.f);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float2 za = r[P + i], zb = r[P + i];
#pragma unroll
        for (int k = 0; k <= i; ++k) {
          const float2 mik = r[tri(i) + k];
          za = __ffma2_rn(mik, xa2[k], za);
          zb = __ffma2_rn(mik, xb2[k], zb);
        }
        sa = __ffma2_rn(make_float2(-za.x, -za.y), za, sa);
        sb = __ffma2_rn(make_float2(-zb.x, -zb.y), zb, sb);
      }
      const float2 ea = ex2_f2(sa), eb = ex2_f2(sb);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float2 wc = r[P + N + c];
        pa[c] = __ffma2_rn(wc, ea, pa[c]);
        pb[c] = __ffma2_rn(wc, eb, pb[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acca[c] = __fadd2_rn(acca[c], pa[c]);
      accb[c] = __fadd2_rn(accb[c], pb[c]);
    }
    __syncthreads();
  }
  if (va) {
#pragma unroll
    for (int c = 0; c < 3; ++c) a.y[(q0 + tid) * 3 + c] = acca[c].x + acca[c].y;
  }
  if (vb) {
#pragma unroll
    for (int c = 0; c < 3; ++c) a.y[(q0 + tid + 128) * 3 + c] = accb[c].x + accb[c].y;
  }
}

// ---- loss ---------------------------------------------------------------------
constexpr int LOSS_BLOCKS = 512;

// Plain L2 (rel_eps < 0): d^2 and dy = scale d.  Relative L2 (rel_eps >= 0,
// Section 4.1's relative L2 read as d^2 / (y^2 + eps) with the denominator
// held constant): d^2 / den and dy = scale d / den.  Per-block partial sums
// in FP64, combined in a fixed order by loss_final_kernel.
template <bool REL>
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ y,
                                                   const float* __restrict__ target,
                                                   float* __restrict__ dy, long long n, double scale,
                                                   double rel_eps, double* __restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double yi = (double)y[i];
    const double d = yi - (double)target[i];
    if (REL) {  // one FP64 division per element (the FP64 rate is low here)
      const double inv = 1.0 / (yi * yi + rel_eps);
      dy[i] = (float)(d * scale * inv);
      acc += d * d * inv;
    } else {
      dy[i] = (float)(d * scale);
      acc += d * d;
    }
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
// One CTA of 128 threads per tile; each thread owns two candidates (the two
// lanes of packed FP32x2 instructions) and loops over the tile's queries,
// read from shared memory as (x - c, dy) duplicated into both lanes.  With
// z' = kappa z: beta = e sum_c dy_c w_c, and the partial record of an entry
// is [sum beta z d^T (lower), sum beta z, sum dy e], formed from
// sum beta z' (x - c)^T - (sum beta z') (m - c)^T at the end.  Records go to
// the entry's Gaussian-major slot slot[c], so that the per-Gaussian sums read
// contiguous memory.  Record: [dl/dM (lower), dl/dm, dl/dw].
template <int N>
__global__ void __launch_bounds__(128) bwd_kernel(BwdArgs a) {
  constexpr int P = tri(N), R = rec_floats(N), R4 = R / 4, RP = part_floats(N);
  constexpr int QS = (2 * (N + 3) + 3) / 4 * 4;  // floats per query: (x - c, dy) x 2 lanes
  __shared__ __align__(16) float sq[NDG_MAX_TILE * QS];
  __shared__ float sred[4 * N * 2];
  __shared__ float sctr[N];
  const long long t = blockIdx.x;
  const int tid = threadIdx.x;
  const long long q0 = t * a.tile;
  const int nq = (int)(a.Q - q0 < a.tile ? a.Q - q0 : a.tile);
  {
    const bool va = tid < nq, vb = tid + 128 < nq;
    float xa[N], xb[N];
#pragma unroll
    for (int d = 0; d < N; ++d) {
      xa[d] = va ? a.x[(q0 + tid) * N + d] : 0.0f;
      xb[d] = vb ? a.x[(q0 + tid + 128) * N + d] : 0.0f;
    }
    tile_centre<N>(xa, va, xb, vb, sred, sctr);
    for (int h = 0; h < 2; ++h) {
      const int qi = tid + 128 * h;
      if (qi >= nq) continue;
      float* row = sq + qi * QS;
#pragma unroll
      for (int d = 0; d < N; ++d) {
        const float v = (h ? xb[d] : xa[d]) - sctr[d];
        row[2 * d] = v;
        row[2 * d + 1] = v;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float v = a.dy[(q0 + qi) * 3 + c];
        row[2 * (N + c)] = v;
        row[2 * (N + c) + 1] = v;
      }
    }
  }
  __syncthreads();
  const long long beg = a.offsets[t], end = a.offsets[t + 1];
  for (long long c0 = beg; c0 < end; c0 += 256) {
    const long long cid[2] = {c0 + tid, c0 + 128 + tid};
    float2 M2[P], b2[N], w2[3];
    float mt[2][N];  // m - c of both candidates (for the final product)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = cid[h] < end ? a.ids[cid[h]] : -1;
      float buf[R];
      if ((unsigned)g < (unsigned)a.Ge) {
        const float4* src = reinterpret_cast<const float4*>(a.rec) + (size_t)g * R4;
#pragma unroll
        for (int i = 0; i < R4; ++i) {
          float4 v = __ldg(src + i);
          buf[4 * i] = v.x; buf[4 * i + 1] = v.y; buf[4 * i + 2] = v.z; buf[4 * i + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int i = 0; i < R; ++i) buf[i] = 0.0f;
      }
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const float v = kKappa * buf[i];
        if (h) M2[i].y = v; else M2[i].x = v;
      }
#pragma unroll
      for (int i = 0; i < N; ++i) mt[h][i] = buf[P + i] - sctr[i];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (h) w2[i].y = buf[P + N + i]; else w2[i].x = buf[P + N + i];
      }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float ba = 0.0f, bb = 0.0f;
#pragma unroll
      for (int k = 0; k <= i; ++k) {
        ba = fmaf(M2[tri(i) + k].x, mt[0][k], ba);
        bb = fmaf(M2[tri(i) + k].y, mt[1][k], bb);
      }
      b2[i] = make_float2(-ba, -bb);
    }
    float2 GM2[P], Gz2[N], Gw2[3];
#pragma unroll
    for (int i = 0; i < P; ++i) GM2[i] = f2(0.f);
#pragma unroll
    for (int i = 0; i < N; ++i) Gz2[i] = f2(0.f);
#pragma unroll
    for (int i = 0; i < 3; ++i) Gw2[i] = f2(0.f);
    for (int qi = 0; qi < nq; ++qi) {
      const float2* qq = reinterpret_cast<const float2*>(sq + qi * QS);
      float2 x2[N], z2[N];
#pragma unroll
      for (int d = 0; d < N; ++d) x2[d] = qq[d];
      float2 s2 = f2(0.f);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float2 z = b2[i];
#pragma unroll
        for (int k = 0; k <= i; ++k) z = __ffma2_rn(M2[tri(i) + k], x2[k], z);
        z2[i] = z;
        s2 = __ffma2_rn(make_float2(-z.x, -z.y), z, s2);
      }
      const float2 e2 = ex2_f2(s2);
      const float2 g0 = qq[N], g1 = qq[N + 1], g2 = qq[N + 2];
      Gw2[0] = __ffma2_rn(g0, e2, Gw2[0]);
      Gw2[1] = __ffma2_rn(g1, e2, Gw2[1]);
      Gw2[2] = __ffma2_rn(g2, e2, Gw2[2]);
      float2 tt = __fmul2_rn(g0, w2[0]);
      tt = __ffma2_rn(g1, w2[1], tt);
      tt = __ffma2_rn(g2, w2[2], tt);
      const float2 beta = __fmul2_rn(e2, tt);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float2 bz = __fmul2_rn(beta, z2[i]);
        Gz2[i] = __fadd2_rn(Gz2[i], bz);
#pragma unroll
        for (int k = 0; k <= i; ++k) GM2[tri(i) + k] = __ffma2_rn(bz, x2[k], GM2[tri(i) + k]);
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (cid[h] >= end) continue;
      // record: dl/dM = -sum beta z d^T (lower), dl/dm = M^T sum beta z, dl/dw
      float buf[RP];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float gz = h ? Gz2[i].y : Gz2[i].x;
#pragma unroll
        for (int k = 0; k <= i; ++k) {
          const float gm = h ? GM2[tri(i) + k].y : GM2[tri(i) + k].x;
          buf[tri(i) + k] = -kInvKappa * fmaf(-gz, mt[h][k], gm);
        }
      }
      constexpr float kInvKappa2 = kInvKappa * kInvKappa;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        float s = 0.0f;
#pragma unroll
        for (int i = k; i < N; ++i) s = fmaf(h ? M2[tri(i) + k].y : M2[tri(i) + k].x,
                                             h ? Gz2[i].y : Gz2[i].x, s);
        buf[P + k] = kInvKappa2 * s;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) buf[P + N + c] = h ? Gw2[c].y : Gw2[c].x;
#pragma unroll
      for (int i = P + N + 3; i < RP; ++i) buf[i] = 0.0f;
      const long long slot = a.slot ? (long long)a.slot[cid[h]] : cid[h];
      float* out = a.part + (size_t)slot * RP;
#pragma unroll
      for (int i = 0; i < RP; i += 4)
        *reinterpret_cast<float4*>(out + i) = make_float4(buf[i], buf[i + 1], buf[i + 2], buf[i + 3]);
    }
  }
}

// ---- per-Gaussian sums of the partial records (Gaussian-major, fixed order) --
// One warp per evaluated Gaussian; its records are positions goff[e] ..
// goff[e+1] of the Gaussian-major order, i.e. records perm[j] (entry order)
// for j in that range (the stable sort keeps entries in tile order).  Lanes
// are split into groups of RP/4 (one float4 column each) that take every
// G-th record; the groups' sums are combined in group order, so the result
// does not depend on scheduling.
__global__ void __launch_bounds__(256) segsum_kernel(const float* __restrict__ part, int RP,
                                                     const long long* __restrict__ goff, int Ge,
                                                     const int32_t* __restrict__ perm,
                                                     long long n_cap, int* status,
                                                     float* __restrict__ gsum) {
  __shared__ float4 sh[8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long e = (long long)blockIdx.x * 8 + warp;
  const int RP4 = RP >> 2;
  const int G = 32 / RP4 > 0 ? 32 / RP4 : 1;
  const int grp = lane / RP4, col = lane - grp * RP4;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (e < Ge && grp < G && col < RP4) {
    // segment bounds and entry indices are kept inside the n_cap records
    // (an order computed for other lists reads no foreign memory)
    long long b = goff[e], en = goff[e + 1];
    b = b < 0 ? 0 : (b > n_cap ? n_cap : b);
    en = en < b ? b : (en > n_cap ? n_cap : en);
    const float4* src = reinterpret_cast<const float4*>(part);
    bool bad = false;
    // four records of the group in flight at a time, added in entry order
    long long j = b + grp;
    for (; j + 3 * G < en; j += 4 * G) {
      long long r[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        r[u] = perm ? (long long)__ldg(perm + j + u * G) : j + u * G;
        if ((unsigned long long)r[u] >= (unsigned long long)n_cap) {
          bad = true;
          r[u] = -1;
        }
      }
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        v[u] = r[u] >= 0 ? __ldg(src + r[u] * RP4 + col) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc.x += v[u].x; acc.y += v[u].y; acc.z += v[u].z; acc.w += v[u].w;
      }
    }
    for (; j < en; j += G) {
      const long long r = perm ? (long long)__ldg(perm + j) : j;
      if ((unsigned long long)r >= (unsigned long long)n_cap) {
        bad = true;
        continue;
      }
      const float4 v = __ldg(src + r * RP4 + col);
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    if (bad && status) set_status(status, NDG_ERR_INVALID_ARG);
  }
  sh[warp][lane] = acc;
  __syncwarp();
  if (e < Ge && lane < RP4) {
    float4 s = sh[warp][lane];
    for (int g = 1; g < G; ++g) {
      const float4 v = sh[warp][g * RP4 + lane];
      s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
    }
    reinterpret_cast<float4*>(gsum)[e * RP4 + lane] = s;
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

// dl/dL (lower) = -M^T (dl/dM) M^T for M = L^-1 (dM = -M dL M).
template <int N>
__device__ __forceinline__ void grad_L(const float* M, const float* GMr, float* GL) {
  float H[N][N];  // H = GMr M^T, H[a][j] = sum_{b <= min(a, j)} GMr[a][b] M[j][b]
#pragma unroll
  for (int aa = 0; aa < N; ++aa)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float s = 0.0f;
#pragma unroll
      for (int b = 0; b <= (aa < j ? aa : j); ++b) s = fmaf(GMr[tri(aa) + b], M[tri(j) + b], s);
      H[aa][j] = s;
    }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      float s = 0.0f;
#pragma unroll
      for (int aa = i; aa < N; ++aa) s = fmaf(M[tri(aa) + i], H[aa][j], s);
      GL[tri(i) + j] = -s;
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

// Record kind 1 to kind 0: dl/dM = 2 M G (lower part; G symmetric, lower
// packed) and dl/dm = 2 A v with A = M^T M.
template <int N>
__device__ __forceinline__ void part_to_dM(const float* M, const float* sp, float* out) {
  constexpr int P = tri(N);
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int k = 0; k <= i; ++k) {
      float s = 0.0f;
#pragma unroll
      for (int l = 0; l <= i; ++l) s = fmaf(M[tri(i) + l], sp[l >= k ? tri(l) + k : tri(k) + l], s);
      out[tri(i) + k] = 2.0f * s;
    }
  float Mv[N];  // M v, then A v = M^T (M v)
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float s = 0.0f;
#pragma unroll
    for (int l = 0; l <= i; ++l) s = fmaf(M[tri(i) + l], sp[P + l], s);
    Mv[i] = s;
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    float s = 0.0f;
#pragma unroll
    for (int i = k; i < N; ++i) s = fmaf(M[tri(i) + k], Mv[i], s);
    out[P + k] = 2.0f * s;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) out[P + N + c] = sp[P + N + c];
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
  float conv[P + N + 3];
  if (a.part_kind == 1) {
    part_to_dM<N>(M, sp, conv);
    sp = conv;
  }
  grad_L<N>(M, sp, GL);
#pragma unroll
  for (int i = 0; i < N; ++i) Gm[i] = sp[P + i];
  if (a.has_children) {
    const float* sc = a.gsum + (size_t)(a.G + g) * RP;
    float U[P], Lc[P], Mc[P], GLc[P], Gmc[N], mu[N], convc[P + N + 3];
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
    if (a.part_kind == 1) {
      part_to_dM<N>(Mc, sc, convc);
      sc = convc;
    }
    grad_L<N>(Mc, sc, GLc);
#pragma unroll
    for (int i = 0; i < N; ++i) Gmc[i] = sc[P + i];
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

// Splits the tiles by candidate count: tiles with at least min_cand
// candidates go to list a, the others to list b (counts in n_a, n_b, zeroed
// by the caller).  The order inside a list does not matter: every tile's
// outputs are computed by one CTA of one kernel.
__global__ void tile_split_kernel(const long long* __restrict__ offsets, long long T,
                                  long long min_cand, int* __restrict__ la, int* __restrict__ lb,
                                  int* __restrict__ n_a, int* __restrict__ n_b) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const bool dense = offsets[t + 1] - offsets[t] >= min_cand;
  if (dense) la[atomicAdd(n_a, 1)] = (int)t;
  else lb[atomicAdd(n_b, 1)] = (int)t;
}

int launch_tile_split(const long long* offsets, long long T, long long min_cand, int* la, int* lb,
                      int* n_a, int* n_b, cudaStream_t s) {
  if (T <= 0) return 0;
  tile_split_kernel<<<(unsigned)ceil_div<long long>(T, 256), 256, 0, s>>>(offsets, T, min_cand, la,
                                                                         lb, n_a, n_b);
  return 1;
}

int launch_fwd(int N, const FwdArgs& a, long long T, cudaStream_t s) {
  if (T <= 0) return 0;
#define L_FWD(n) fwd_kernel<n><<<(unsigned)T, 128, 0, s>>>(a)
  NDG_SWITCH_N(N, L_FWD)
#undef L_FWD
  return 1;
}

int launch_loss(const float* y, const float* target, float* dy, long long n, double* part,
                double* loss, cudaStream_t s, double rel_eps, long long norm) {
  if (norm <= 0) norm = n;  // the mean over these n outputs, or over a larger set
  const double scale = norm > 0 ? 2.0 / (double)norm : 0.0;
  if (rel_eps >= 0.0)
    loss_kernel<true><<<LOSS_BLOCKS, 256, 0, s>>>(y, target, dy, n, scale, rel_eps, part);
  else
    loss_kernel<false><<<LOSS_BLOCKS, 256, 0, s>>>(y, target, dy, n, scale, rel_eps, part);
  loss_final_kernel<<<1, LOSS_BLOCKS, 0, s>>>(part, norm, loss);
  return 2;
}

int launch_bwd(int N, const BwdArgs& a, long long T, cudaStream_t s) {
  if (T <= 0) return 0;
#define L_BWD(n) bwd_kernel<n><<<(unsigned)T, 128, 0, s>>>(a)
  NDG_SWITCH_N(N, L_BWD)
#undef L_BWD
  return 1;
}

int launch_segsum(const float* part, int RP, const long long* goff, int Ge, const int32_t* perm,
                  long long n_cap, int* status, float* gsum, cudaStream_t s) {
  if (Ge <= 0) return 0;
  segsum_kernel<<<(unsigned)ceil_div<long long>(Ge, 8), 256, 0, s>>>(part, RP, goff, Ge, perm,
                                                                    n_cap, status, gsum);
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
