// cull.cu -- parameter preparation and the random-projection cull
// (Section 3.2, Eq. 3-5) behind ndg_build_cull.
//
// Pipeline (one stream, no host synchronisation):
//   tile_bounds   per tile and projection: min / max of q^T r_j (FP32 fmaf
//                 chain), one warp per tile
//   cull_range    per projection: global min / max over tiles and the bucket
//                 scale inv_h_j = B / (hi_j - lo_j)
//   tile_keys     per tile and projection: bucket range [tlo, thi] (bytes)
//   prep          per evaluated Gaussian: FP64 activation (Eq. 2, 6-8), the
//                 prepared record (M = L^{-1}, m, w) and the bucket range of
//                 [m_r - k_g sigma_r, m_r + k_g sigma_r] for every projection
//                 (bytes), plus its first-projection bin blo * B + bhi
//   radix sort    Gaussians by bin (stable, so ascending index inside a bin)
//   cull_tile     one CTA per tile visits exactly the Gaussians whose first
//                 projection range meets the tile's: bins (b, >= tlo) for
//                 b <= thi are contiguous runs of the sorted order; the other
//                 projections are tested four at a time with byte-SIMD
//                 compares; survivors are compacted with warp ballots and a
//                 block prefix.  Run twice: count, then (after a scan of the
//                 counts) fill.
#include "common.cuh"
#include "internal.h"
#include "kernels.h"

namespace ndg {

// ---- tile bounds ----------------------------------------------------------
template <int N>
__global__ void tile_bounds_kernel(const float* __restrict__ x, long long Q, int tile, long long T,
                                   int k, const float* __restrict__ proj, float* __restrict__ tb,
                                   int nd) {
  const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= T) return;
  const long long q0 = t * tile;
  const long long q1 = q0 + tile < Q ? q0 + tile : Q;
  for (int j = 0; j < k; ++j) {
    float pj[N];
#pragma unroll
    for (int d = 0; d < N; ++d) pj[d] = proj[j * N + d];
    float lo = INFINITY, hi = -INFINITY;
    for (long long q = q0 + lane; q < q1; q += 32) {
      float acc = 0.0f;
#pragma unroll
      for (int d = 0; d < N; ++d)
        if (d < nd) acc = __fmaf_rn(x[q * N + d], pj[d], acc);  // nd = 3: position only
      lo = fminf(lo, acc);
      hi = fmaxf(hi, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      tb[(t * k + j) * 2 + 0] = lo;
      tb[(t * k + j) * 2 + 1] = hi;
    }
  }
}

// ---- global range per projection ------------------------------------------
// range layout: lo[NDG_MAX_K], hi[NDG_MAX_K], inv_h[NDG_MAX_K]
__global__ void cull_range_kernel(const float* __restrict__ tb, long long T, int k, int B,
                                  long long Q, float* __restrict__ range) {
  __shared__ float slo[256], shi[256];
  for (int j = 0; j < k; ++j) {
    float lo = INFINITY, hi = -INFINITY;
    for (long long t = threadIdx.x; t < T; t += blockDim.x) {
      lo = fminf(lo, tb[(t * k + j) * 2 + 0]);
      hi = fmaxf(hi, tb[(t * k + j) * 2 + 1]);
    }
    slo[threadIdx.x] = lo;
    shi[threadIdx.x] = hi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        slo[threadIdx.x] = fminf(slo[threadIdx.x], slo[threadIdx.x + s]);
        shi[threadIdx.x] = fmaxf(shi[threadIdx.x], shi[threadIdx.x + s]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      float l = slo[0], h = shi[0];
      float rng = __fsub_rn(h, l);
      float mag = fabsf(l) > fabsf(h) ? fabsf(l) : fabsf(h);
      float ih = 0.0f;
      if (Q > 0 && rng > __fmul_rn(1e-3f, __fadd_rn(1.0f, mag))) ih = __fdiv_rn((float)B, rng);
      range[j] = l;
      range[NDG_MAX_K + j] = h;
      range[2 * NDG_MAX_K + j] = ih;
    }
    __syncthreads();
  }
}

// ---- tile bucket keys ---------------------------------------------------------
// tkey row per tile: KP low bytes then KP high bytes; padding projections
// are [0, 255] so they never reject.
__global__ void tile_keys_kernel(const float* __restrict__ tb, long long T, int k, int KP, int B,
                                 const float* __restrict__ range, uint8_t* __restrict__ tkey) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T * KP) return;
  long long t = i / KP;
  int j = (int)(i % KP);
  uint8_t lo = 0, hi = 255;
  if (j < k) {
    float l = range[j], ih = range[2 * NDG_MAX_K + j];
    lo = (uint8_t)clampi(bucket_raw(tb[(t * k + j) * 2 + 0], l, ih, B), 0, B - 1);
    hi = (uint8_t)clampi(bucket_raw(tb[(t * k + j) * 2 + 1], l, ih, B), 0, B - 1);
  }
  tkey[t * 2 * KP + j] = lo;
  tkey[t * 2 * KP + KP + j] = hi;
}

// ---- prep: activation, prepared record, Gaussian keys --------------------------
// Section 3.1 (Eq. 2): L_ii = exp(theta_ii), L_ij = 2 sigmoid(theta_ij) - 1;
// evaluated in FP64 and rounded once to FP32 so that the FP32 values that
// feed the cull contract are the correctly rounded activations.
template <int N>
__device__ __forceinline__ void act_lower64(const float* __restrict__ th, double* L) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      double v = (double)th[tri(i) + j];
      L[tri(i) + j] = (i == j) ? exp(v) : 2.0 / (1.0 + exp(-v)) - 1.0;
    }
}

// Section 3.2 conditioning of one Gaussian on the constant inputs xc beyond
// position, in FP64 with separately rounded products and sums (no fused
// multiply-add), in the order of the plain definition: M = L^-1,
// A = M^T M, d_c = xc - m_c, b = A_pc d_c, C C^T = A_pp (Cholesky),
// z = A_pp^-1 b, q_c = d_c^T A_cc d_c - b^T z; the restriction is
// wc = w exp(-q_c / 2) times a 3-D Gaussian with mean mu = m_p - z and
// covariance T^T T, T = C^-1.  Outputs rounded once to FP32.
template <int N>
__device__ bool condition_gaussian(const double* L, const double* m, const float* wf,
                                   const float* __restrict__ xc, float* muf, float* Tf, float* wcf) {
  double M[N][N], A[N][N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
#pragma unroll
    for (int i = 0; i < N; ++i) M[i][j] = 0.0;
    M[j][j] = __ddiv_rn(1.0, L[tri(j) + j]);
#pragma unroll
    for (int i = j + 1; i < N; ++i) {
      double s = 0.0;
#pragma unroll
      for (int k = j; k < i; ++k) s = __dadd_rn(s, __dmul_rn(L[tri(i) + k], M[k][j]));
      M[i][j] = __ddiv_rn(-s, L[tri(i) + i]);
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < N; ++k) s = __dadd_rn(s, __dmul_rn(M[k][i], M[k][j]));
      A[i][j] = s;
    }
  double dc[N], b[3];
#pragma unroll
  for (int i = 3; i < N; ++i) dc[i] = __dsub_rn((double)xc[i - 3], m[i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
#pragma unroll
    for (int k = 3; k < N; ++k) s = __dadd_rn(s, __dmul_rn(A[i][k], dc[k]));
    b[i] = s;
  }
  double C[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      double s = A[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) s = __dsub_rn(s, __dmul_rn(C[i][k], C[j][k]));
      C[i][j] = (i == j) ? __dsqrt_rn(s) : __ddiv_rn(s, C[j][j]);
    }
  double y3[3], z[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double s = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s = __dsub_rn(s, __dmul_rn(C[i][k], y3[k]));
    y3[i] = __ddiv_rn(s, C[i][i]);
  }
#pragma unroll
  for (int i = 2; i >= 0; --i) {
    double s = y3[i];
#pragma unroll
    for (int k = i + 1; k < 3; ++k) s = __dsub_rn(s, __dmul_rn(C[k][i], z[k]));
    z[i] = __ddiv_rn(s, C[i][i]);
  }
  double qc = 0.0;
#pragma unroll
  for (int i = 3; i < N; ++i) {
    double s = 0.0;
#pragma unroll
    for (int k = 3; k < N; ++k) s = __dadd_rn(s, __dmul_rn(A[i][k], dc[k]));
    qc = __dadd_rn(qc, __dmul_rn(dc[i], s));
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) qc = __dsub_rn(qc, __dmul_rn(b[i], z[i]));
  const double f = exp(__dmul_rn(-0.5, qc));
  bool finite = true;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    muf[i] = (float)__dsub_rn(m[i], z[i]);
    wcf[i] = (float)__dmul_rn((double)wf[i], f);
    finite &= isfinite(muf[i]) && isfinite(wcf[i]);
  }
  double T[3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
#pragma unroll
    for (int i = 0; i < 3; ++i) T[i][j] = 0.0;
    T[j][j] = __ddiv_rn(1.0, C[j][j]);
#pragma unroll
    for (int i = j + 1; i < 3; ++i) {
      double s = 0.0;
#pragma unroll
      for (int k = j; k < i; ++k) s = __dadd_rn(s, __dmul_rn(C[i][k], T[k][j]));
      T[i][j] = __ddiv_rn(-s, C[i][i]);
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Tf[i * 3 + j] = (float)T[i][j];
      finite &= isfinite(Tf[i * 3 + j]);
    }
  return finite;
}

template <int N>
__global__ void __launch_bounds__(128) prep_kernel(PrepArgs a) {
  constexpr int P = tri(N);
  constexpr int R = rec_floats(N);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.Ge) return;
  const bool child = e >= a.G;
  const int g = child ? e - a.G : e;
  double L[P], m[N];
  act_lower64<N>(a.theta + (size_t)g * P, L);
#pragma unroll
  for (int i = 0; i < N; ++i) m[i] = (double)a.mean[(size_t)g * N + i];
  double araw;
  const float* gam;
  if (child) {
    // Section 3.3, Eq. 6-7: L_c = L_p U, m_c = L_p m_u + m_p
    double U[P], Lc[P], mc[N];
    act_lower64<N>(a.u_theta + (size_t)g * P, U);
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
      for (int j = 0; j <= i; ++j) {
        double s = 0.0;
#pragma unroll
        for (int kk = j; kk <= i; ++kk) s = fma(L[tri(i) + kk], U[tri(kk) + j], s);
        Lc[tri(i) + j] = s;
      }
      double s = 0.0;
#pragma unroll
      for (int kk = 0; kk <= i; ++kk) s = fma(L[tri(i) + kk], (double)a.m_u[(size_t)g * N + kk], s);
      mc[i] = s + m[i];
    }
#pragma unroll
    for (int i = 0; i < P; ++i) L[i] = Lc[i];
#pragma unroll
    for (int i = 0; i < N; ++i) m[i] = mc[i];
    araw = (double)a.c_alpha_raw[g];
    gam = a.c_color_raw + (size_t)g * 3;
  } else {
    araw = (double)a.alpha_raw[g];
    gam = a.color_raw + (size_t)g * 3;
  }
  // Section 4.1 (Eq. 8): w = exp(a) sigmoid(gamma)
  const double alpha = exp(araw);
  float wf[3];
  bool finite = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    wf[c] = (float)(alpha * (1.0 / (1.0 + exp(-(double)gam[c]))));
    finite &= isfinite(wf[c]);
  }
  float Lf[P], mf[N];
#pragma unroll
  for (int i = 0; i < P; ++i) { Lf[i] = (float)L[i]; finite &= isfinite(Lf[i]); }
#pragma unroll
  for (int i = 0; i < N; ++i) { mf[i] = (float)m[i]; finite &= isfinite(mf[i]); }
  if (!finite && a.status) set_status(a.status, NDG_ERR_NUMERIC);

  if (a.rec) {
    // M = L^{-1} (lower) by forward substitution on the identity, in FP64.
    double M[P];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      M[tri(j) + j] = 1.0 / L[tri(j) + j];
#pragma unroll
      for (int i = j + 1; i < N; ++i) {
        double s = 0.0;
#pragma unroll
        for (int kk = j; kk < i; ++kk) s = fma(L[tri(i) + kk], M[tri(kk) + j], s);
        M[tri(i) + j] = -s / L[tri(i) + i];
      }
    }
    float* out = a.rec + (size_t)e * (a.rec_kind == 2 ? rec_tc_floats(N) : R);
    float buf[R];
    if (a.rec_kind >= 1) {
      // A = V^-1 = M^T M (lower, packed): A_ij = sum_{k >= i} M_ki M_kj, j <= i
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
          double s = 0.0;
#pragma unroll
          for (int kk = i; kk < N; ++kk) s = fma(M[tri(kk) + i], M[tri(kk) + j], s);
          buf[tri(i) + j] = (float)s;
        }
    } else {
#pragma unroll
      for (int i = 0; i < P; ++i) buf[i] = (float)M[i];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) buf[P + i] = mf[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) buf[P + N + c] = wf[c];
#pragma unroll
    for (int i = P + N + 3; i < R; ++i) buf[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < R; i += 4)
      *reinterpret_cast<float4*>(out + i) = make_float4(buf[i], buf[i + 1], buf[i + 2], buf[i + 3]);
    if (a.rec_kind == 2) {
      constexpr int PM = (P + 3) / 4 * 4;
      float mb[PM];
#pragma unroll
      for (int i = 0; i < PM; ++i) mb[i] = i < P ? (float)M[i] : 0.0f;
#pragma unroll
      for (int i = 0; i < PM; i += 4)
        *reinterpret_cast<float4*>(out + R + i) = make_float4(mb[i], mb[i + 1], mb[i + 2], mb[i + 3]);
    }
  }

  if (a.gkey || a.bin) {
    // conditioned keys: the Gaussian restricted to the constant inputs
    float cmu[3], cT[9], cw[3];
    const bool cond = a.xc != nullptr;
    bool live = finite;
    if constexpr (N >= 4) {
      if (cond) live = live && condition_gaussian<N>(L, m, wf, a.xc, cmu, cT, cw);
    }
    // Cull radius: k_sigma, or sqrt(2 ln(w_max / cutoff)) from the FP32
    // weights (conditioned: the conditional weights) in FP64, rounded once;
    // a child keeps at least child_k_min (Section 3.3: it is optimised while
    // negligible), also below the cutoff.
    float kg;
    bool reach = true;
    if (a.cutoff > 0.0f) {
      float wm = cond ? fmaxf(fmaxf(cw[0], cw[1]), cw[2]) : fmaxf(fmaxf(wf[0], wf[1]), wf[2]);
      if (wm > a.cutoff) kg = (float)sqrt(2.0 * log((double)wm / (double)a.cutoff));
      else { kg = -1.0f; reach = false; }
    } else {
      kg = a.k_sigma;
    }
    if (child && a.child_k_min > 0.0f && a.child_k_min > kg) {
      kg = a.child_k_min;
      reach = true;
    }
    live = live && reach;
    uint8_t klo[NDG_MAX_K], khi[NDG_MAX_K];
    int blo0 = 0, bhi0 = 0;
    for (int j = 0; j < a.k && live; ++j) {
      const float* r = a.proj + j * N;
      float rr[N];
#pragma unroll
      for (int d = 0; d < N; ++d) rr[d] = r[d];
      float mr = 0.0f, s2 = 0.0f;
      if (cond) {  // position only: m_r = mu . r, sigma_r^2 = |T r|^2
#pragma unroll
        for (int d = 0; d < 3; ++d) mr = __fmaf_rn(cmu[d], rr[d], mr);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          float tc = 0.0f;
#pragma unroll
          for (int c = 0; c <= i; ++c) tc = __fmaf_rn(cT[i * 3 + c], rr[c], tc);
          s2 = __fmaf_rn(tc, tc, s2);
        }
      } else {
#pragma unroll
        for (int d = 0; d < N; ++d) mr = __fmaf_rn(mf[d], rr[d], mr);
#pragma unroll
        for (int c = 0; c < N; ++c) {
          float tc = 0.0f;
#pragma unroll
          for (int i = c; i < N; ++i) tc = __fmaf_rn(Lf[tri(i) + c], rr[i], tc);
          s2 = __fmaf_rn(tc, tc, s2);
        }
      }
      const float sr = __fsqrt_rn(s2);
      const float ks = __fmul_rn(kg, sr);
      const float lo = a.range[j], ih = a.range[2 * NDG_MAX_K + j];
      int blo = bucket_raw(__fsub_rn(mr, ks), lo, ih, a.B) - 1;
      int bhi = bucket_raw(__fadd_rn(mr, ks), lo, ih, a.B) + 1;
      if (bhi < 0 || blo > a.B - 1) { live = false; break; }
      blo = blo < 0 ? 0 : blo;
      bhi = bhi > a.B - 1 ? a.B - 1 : bhi;
      klo[j] = (uint8_t)blo;
      khi[j] = (uint8_t)bhi;
      if (j == 0) { blo0 = blo; bhi0 = bhi; }
    }
    if (a.gkey) {
      uint8_t* row = a.gkey + (size_t)e * 2 * a.KP;
      for (int j = 0; j < a.KP; ++j) {
        uint8_t lo = 0, hi = 255;
        if (!live) { lo = 255; hi = 0; }
        else if (j < a.k) { lo = klo[j]; hi = khi[j]; }
        row[j] = lo;
        row[a.KP + j] = hi;
      }
    }
    if (a.bin) {
      const int nb = a.k > 0 ? a.B : 1;
      a.bin[e] = live ? (uint32_t)(blo0 * nb + bhi0) : (uint32_t)(nb * nb);
    }
  }
}

// ---- per-tile candidate lists ----------------------------------------------------
__device__ __forceinline__ bool keys_overlap(const uint32_t* glo, const uint32_t* ghi,
                                             const uint32_t* tlo, const uint32_t* thi, int words) {
  uint32_t ok = 0xffffffffu;
  for (int w = 0; w < words; ++w)
    ok &= __vcmpleu4(glo[w], thi[w]) & __vcmpleu4(tlo[w], ghi[w]);
  return ok == 0xffffffffu;
}

// One CTA of CT_WARPS warps per tile.  The tile's sources (Gaussians whose
// first-projection bucket range meets the tile's) are thi0 + 1 runs of the
// bin-sorted order; warp w takes the contiguous slice w of their
// concatenation (slice bounds at multiples of 32), walks it 32 elements at
// a time (each lane tracks its run).  The count pass tests the remaining
// projections, counts the survivors and stores the ballot of every 32
// sources in masks[t][i / 32]; the fill pass reads the ballots back (no
// key loads) and writes the survivors in order at the scanned offset of
// (tile, warp), so the list order is the concatenation order.
template <int KP>
__global__ void __launch_bounds__(256) cull_tile_kernel(CullTileArgs a) {
  constexpr int W = KP / 4;  // 32-bit words per key half (KP >= 8)
  __shared__ long long rbeg[256];
  __shared__ long long rpre[257];
  __shared__ long long s_total;
  __shared__ long long ws_[8];
  const long long t = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t tlo[W > 0 ? W : 1], thi[W > 0 ? W : 1];
  int tlo0 = 0, thi0 = 0;
  if (KP > 0) {
    const uint32_t* tk = reinterpret_cast<const uint32_t*>(a.tkey + t * 2 * KP);
#pragma unroll
    for (int w = 0; w < W; ++w) { tlo[w] = tk[w]; thi[w] = tk[W + w]; }
    tlo0 = a.tkey[t * 2 * KP];
    thi0 = a.tkey[t * 2 * KP + KP];
  }
  const int nb = KP > 0 ? a.B : 1;
  const int nr = thi0 + 1;  // first-projection bucket rows b = 0 .. thi0
  {
    long long len = 0;
    if (tid < nr) {
      long long b0 = a.binoff[(long long)tid * nb + tlo0];
      long long b1 = a.binoff[(long long)(tid + 1) * nb];
      rbeg[tid] = b0;
      len = b1 > b0 ? b1 - b0 : 0;
    }
    long long v = tid < nr ? len : 0, incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) ws_[warp] = incl;
    __syncthreads();
    long long off = 0;
    for (int w = 0; w < warp; ++w) off += ws_[w];
    if (tid < nr) rpre[tid] = incl - v + off;
    if (tid == 255) rpre[nr] = incl + off;  // total (threads past nr add 0)
    __syncthreads();
    if (tid == 0) s_total = rpre[nr];
    __syncthreads();
  }
  const long long n_src = s_total;
  auto bound = [&](int w) -> long long {
    const long long v = (n_src * w / 8 + 31) / 32 * 32;
    return v < n_src ? v : n_src;
  };
  const long long lo = bound(warp), hi = warp == 7 ? n_src : bound(warp + 1);
  uint32_t* masks = a.masks + t * a.mask_words;
  // run of the slice's first element: largest r with rpre[r] <= lo
  int r = 0;
  {
    int a0 = 0, b0 = nr - 1;
    while (a0 < b0) {
      int mid = (a0 + b0 + 1) >> 1;
      if (rpre[mid] <= lo) a0 = mid; else b0 = mid - 1;
    }
    r = a0;
  }
  const bool fill = a.ids != nullptr;
  long long written = fill ? a.excl[t * 8 + warp] : 0;
  long long count = 0;
  for (long long i0 = lo; i0 < hi; i0 += 32) {
    const long long i = i0 + lane;
    unsigned bal;
    if (!fill) {
      bool pass = false;
      if (i < hi) {
        if (KP > 0) {
          while (r + 1 < nr && rpre[r + 1] <= i) ++r;
          const long long pos = rbeg[r] + (i - rpre[r]);
          // keys in bin-sorted order: a warp reads consecutive rows, 16 bytes
          // per load (rows are 2 KP = 16, 32, 48 or 64 bytes, 16-byte aligned)
          const uint4* gk = reinterpret_cast<const uint4*>(a.gkey + (size_t)pos * 2 * KP);
          uint32_t row[2 * W > 4 ? 2 * W : 4];
#pragma unroll
          for (int v = 0; v < (2 * W) / 4; ++v) {
            const uint4 q = __ldg(gk + v);
            row[4 * v] = q.x; row[4 * v + 1] = q.y; row[4 * v + 2] = q.z; row[4 * v + 3] = q.w;
          }
          pass = keys_overlap(row, row + W, tlo, thi, W);
        } else {
          pass = true;
        }
      }
      bal = __ballot_sync(0xffffffffu, pass);
      if (lane == 0) masks[i0 >> 5] = bal;
    } else {
      bal = masks[i0 >> 5];
      if ((bal >> lane) & 1u) {
        while (r + 1 < nr && rpre[r + 1] <= i) ++r;
        const long long src = rbeg[r] + (i - rpre[r]);
        const long long pos = written + count + __popc(bal & ((1u << lane) - 1u));
        if (pos < a.E_cap) a.ids[pos] = a.sorted_ids[src];
      }
    }
    count += __popc(bal);
  }
  if (!fill && lane == 0) a.counts[t * 8 + warp] = count;
}

// Key rows in bin-sorted order: dst[p] = src[sorted[p]] (2 KP bytes a row).
__global__ void permute_keys_kernel(const uint8_t* __restrict__ src, const int32_t* __restrict__ sorted,
                                    int n, int row_words, uint32_t* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * row_words) return;
  const long long p = i / row_words;
  const int w = (int)(i - p * row_words);
  dst[i] = reinterpret_cast<const uint32_t*>(src + (size_t)sorted[p] * row_words * 4)[w];
}

// ---- launchers ------------------------------------------------------------------
#define NDG_CASE_N(n, call) case n: call(n); break;
#define NDG_SWITCH_N(N, call)                                                         \
  switch (N) {                                                                        \
    NDG_CASE_N(1, call) NDG_CASE_N(2, call) NDG_CASE_N(3, call) NDG_CASE_N(4, call)   \
    NDG_CASE_N(5, call) NDG_CASE_N(6, call) NDG_CASE_N(7, call) NDG_CASE_N(8, call)   \
    NDG_CASE_N(9, call) NDG_CASE_N(10, call) NDG_CASE_N(11, call) NDG_CASE_N(12, call) \
    default: break;                                                                   \
  }

int launch_tile_bounds(int N, const float* x, long long Q, int tile, long long T, int k,
                       const float* proj, float* tb, cudaStream_t s, int nd) {
  if (T <= 0 || k <= 0) return 0;
  if (nd <= 0 || nd > N) nd = N;
  unsigned blocks = (unsigned)ceil_div<long long>(T * 32, 256);
#define L_TB(n) tile_bounds_kernel<n><<<blocks, 256, 0, s>>>(x, Q, tile, T, k, proj, tb, nd)
  NDG_SWITCH_N(N, L_TB)
#undef L_TB
  return 1;
}

int launch_cull_range(const float* tb, long long T, int k, int B, long long Q, float* range,
                      cudaStream_t s) {
  if (k <= 0) return 0;
  cull_range_kernel<<<1, 256, 0, s>>>(tb, T, k, B, Q, range);
  return 1;
}

int launch_tile_keys(const float* tb, long long T, int k, int KP, int B, const float* range,
                     uint8_t* tkey, cudaStream_t s) {
  if (T <= 0 || KP <= 0) return 0;
  tile_keys_kernel<<<(unsigned)ceil_div<long long>(T * KP, 256), 256, 0, s>>>(tb, T, k, KP, B,
                                                                             range, tkey);
  return 1;
}

int launch_prep(int N, const PrepArgs& a, cudaStream_t s) {
  if (a.Ge <= 0) return 0;
  unsigned blocks = (unsigned)ceil_div(a.Ge, 128);
#define L_PREP(n) prep_kernel<n><<<blocks, 128, 0, s>>>(a)
  NDG_SWITCH_N(N, L_PREP)
#undef L_PREP
  return 1;
}

int launch_permute_keys(const uint8_t* src, const int32_t* sorted, int n, int KP, uint8_t* dst,
                        cudaStream_t s) {
  if (n <= 0 || KP <= 0) return 0;
  const int row_words = 2 * KP / 4;
  permute_keys_kernel<<<(unsigned)ceil_div<long long>((long long)n * row_words, 256), 256, 0, s>>>(
      src, sorted, n, row_words, reinterpret_cast<uint32_t*>(dst));
  return 1;
}

int launch_cull_tile(int KP, const CullTileArgs& a, long long T, cudaStream_t s) {
  if (T <= 0) return 0;
  switch (KP) {
    case 0: cull_tile_kernel<0><<<(unsigned)T, 256, 0, s>>>(a); break;
    case 8: cull_tile_kernel<8><<<(unsigned)T, 256, 0, s>>>(a); break;
    case 16: cull_tile_kernel<16><<<(unsigned)T, 256, 0, s>>>(a); break;
    case 24: cull_tile_kernel<24><<<(unsigned)T, 256, 0, s>>>(a); break;
    case 32: cull_tile_kernel<32><<<(unsigned)T, 256, 0, s>>>(a); break;
    default: return 0;
  }
  return 1;
}

}  // namespace ndg
