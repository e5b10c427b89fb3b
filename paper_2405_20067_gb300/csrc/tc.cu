// tc.cu -- the lifted-feature evaluation on the 5th-generation tensor cores
// (tcgen05, TMEM accumulator) behind ndg_forward(NDG_MODE_TC).
//
// The exponent of Eq. 1 is a quadratic form, so for a tile with centre c,
// x~ = x - c and m~ = m - c, with A = V^-1 = M^T M:
//   s = x~^T A x~ - 2 (A m~)^T x~ + m~^T A m~ = phi(x~) . coef
// with lifted query features phi = [x~_i x~_j (j <= i), x~_i, 1] (F = P + N + 1)
// and per-(Gaussian, tile) coefficients coef = [A_ii | 2 A_ij, -2 A m~, m~^T A m~],
// here pre-multiplied by -log2(e)/2 so that the accumulator holds log2 of the
// Gaussian factor.  For every chunk of NC candidates of a tile the CTA
// computes the 128 x NC matrix  S = Phi Coef^T  with tcgen05.mma kind::tf32:
// operands are split into TF32 high and low parts and three products
// (hi hi + hi lo + lo hi) are accumulated in FP32 in tensor memory, which
// keeps ~21 bits of the products (the centring keeps the cancellation between
// the quadratic, linear and constant terms small).  The epilogue reads S
// from TMEM (tcgen05.ld), forms e = 2^S on the MUFU and accumulates w e with
// packed FP32x2 FMAs.
//
// CTA: 128 threads = 4 warps; thread i owns query row i of the M = 128 block
// (TMEM lane i); a 256-query tile is handled by two CTAs.  Shared memory
// (no swizzle, K-major canonical layout: 8-row x 16-byte core matrices,
// core matrices along K at LBO = 128 B, 8-row groups at SBO = KP/4 * 128 B):
// Phi_hi, Phi_lo [128 x KP], Coef_hi, Coef_lo [NC x KP], w [NC] float4.
// Every wait on the MMA completion barrier is bounded; a timeout sets
// NDG_ERR_TIMEOUT, waits (bounded) once more, frees TMEM and exits.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "kernels.h"
#include "tcgen05.cuh"

namespace ndg {


template <int N>
struct TcShape {
  static constexpr int P = tri(N);
  static constexpr int F = P + N + 1;
  static constexpr int KP = (F + 7) / 8 * 8;
  static constexpr int NC = N <= 8 ? 128 : 64;  // candidates per MMA (the N dimension)
  static constexpr uint32_t SBO_A = (KP / 4) * 128;
  static constexpr uint32_t SBO_B = (KP / 4) * 128;
  static constexpr uint32_t A_BYTES = 128u * KP * 4;
  static constexpr uint32_t B_BYTES = (uint32_t)NC * KP * 4;
  static constexpr uint32_t W_BYTES = (uint32_t)NC * 16;  // pairs: w0 w0' w1 w1' w2 w2' - -
  static constexpr uint32_t TMEM_COLS = 2 * NC;          // two accumulators
  static constexpr uint32_t SMEM_USED = 2 * A_BYTES + 2 * (2 * B_BYTES + W_BYTES) + 128;
  // at most 512 / TMEM_COLS CTAs may share an SM's tensor memory: request
  // enough shared memory that no more than that many are resident
  static constexpr uint32_t SMEM_FLOOR = (228u * 1024u) / (512u / TMEM_COLS + 1) + 1024u;
  static constexpr uint32_t SMEM = SMEM_USED > SMEM_FLOOR ? SMEM_USED : SMEM_FLOOR;
  static_assert(SMEM <= 227u * 1024u, "shared memory");
};

// Loads the prepared record of candidate j of a chunk (zeros past the end or
// for an index outside the mixture).
template <int N>
__device__ __forceinline__ void load_record(const FwdArgs& a, long long c0, int n, int j,
                                            float4 (&rec)[rec_floats(N) / 4]) {
  constexpr int R4 = rec_floats(N) / 4;
  const int g = j < n ? a.ids[c0 + j] : -1;
  if ((unsigned)g < (unsigned)a.Ge) {
    const float4* src = reinterpret_cast<const float4*>(a.rec) + (size_t)g * R4;
#pragma unroll
    for (int i = 0; i < R4; ++i) rec[i] = __ldg(src + i);
  } else {
#pragma unroll
    for (int i = 0; i < R4; ++i) rec[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Stages candidate j from its record (A packed, m, w; all zero for a
// padding slot): coefficient row (split hi / lo) into the Coef buffers and
// its weights into the packed pair array.
template <int N>
__device__ __forceinline__ void stage_coef(const float4 (&rec)[rec_floats(N) / 4], int j,
                                           const float* __restrict__ sctr, uint8_t* Bhi,
                                           uint8_t* Blo, float* sw2) {
  using S = TcShape<N>;
  constexpr int P = S::P, KP = S::KP, R = rec_floats(N), R4 = R / 4;
  float buf[R];
#pragma unroll
  for (int i = 0; i < R4; ++i) {
    buf[4 * i] = rec[i].x; buf[4 * i + 1] = rec[i].y; buf[4 * i + 2] = rec[i].z; buf[4 * i + 3] = rec[i].w;
  }
  const bool live = buf[P + N] != 0.0f || buf[P + N + 1] != 0.0f || buf[P + N + 2] != 0.0f ||
                    buf[0] != 0.0f;
  float coef[KP];
  float mt[N];
#pragma unroll
  for (int i = 0; i < N; ++i) mt[i] = live ? buf[P + i] - sctr[i] : 0.0f;
  float cst = 0.0f;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < N; ++k) s = fmaf(buf[i >= k ? tri(i) + k : tri(k) + i], mt[k], s);
    coef[P + i] = kNegHalfLog2eTC * (-2.0f * s);
    cst = fmaf(mt[i], s, cst);
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int k = 0; k <= i; ++k)
      coef[tri(i) + k] = kNegHalfLog2eTC * (i == k ? buf[tri(i) + k] : 2.0f * buf[tri(i) + k]);
  coef[P + N] = kNegHalfLog2eTC * cst;
#pragma unroll
  for (int k = P + N + 1; k < KP; ++k) coef[k] = 0.0f;
  store_row_split<KP>(Bhi, Blo, j, S::SBO_B, coef);
  float* d = sw2 + (j >> 1) * 8 + (j & 1);
  d[0] = buf[P + N];
  d[2] = buf[P + N + 1];
  d[4] = buf[P + N + 2];
}

template <int N>
__global__ void __launch_bounds__(128) fwd_tc_kernel(FwdArgs a) {
  using S = TcShape<N>;
  constexpr int P = S::P, KP = S::KP, NC = S::NC;
  extern __shared__ __align__(128) uint8_t dsm[];
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm + 127) & ~(uintptr_t)127);
  uint8_t* Ahi = base;
  uint8_t* Alo = Ahi + S::A_BYTES;
  uint8_t* Bbuf = Alo + S::A_BYTES;  // two stages of (Bhi, Blo, w)
  constexpr uint32_t STAGE = 2 * S::B_BYTES + S::W_BYTES;
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ float sred[4 * N * 2];
  __shared__ float sctr[N];
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5;
  const int halves = (a.tile + 127) >> 7;
  const long long t = blockIdx.x / halves;
  const int half = blockIdx.x - (int)(t * halves);
  const long long qt = t * a.tile;  // first query of the tile
  const long long q0 = qt + half * 128;
  const long long qend_tile = qt + a.tile < a.Q ? qt + a.tile : a.Q;
  const int nq = (int)(qend_tile - q0 < 128 ? qend_tile - q0 : 128);
  const bool active = tid < nq;

  // queries, centre, lifted features (row tid of Phi)
  float xq[N], dummy[N];
#pragma unroll
  for (int d = 0; d < N; ++d) {
    xq[d] = active ? a.x[(q0 + tid) * N + d] : 0.0f;
    dummy[d] = 0.0f;
  }
  tile_centre<N>(xq, active, dummy, false, sred, sctr);
  {
    float xt[N];
#pragma unroll
    for (int d = 0; d < N; ++d) xt[d] = active ? xq[d] - sctr[d] : 0.0f;
    float phi[KP];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) phi[tri(i) + j] = xt[i] * xt[j];
#pragma unroll
    for (int i = 0; i < N; ++i) phi[P + i] = xt[i];
    phi[P + N] = active ? 1.0f : 0.0f;
#pragma unroll
    for (int k = P + N + 1; k < KP; ++k) phi[k] = 0.0f;
    store_row_split<KP>(Ahi, Alo, tid, S::SBO_A, phi);
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, S::TMEM_COLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const long long beg = a.offsets[t], end = a.offsets[t + 1];
  const int nchunks = (int)((end - beg + NC - 1) / NC);
  auto chunk_n = [&](int i) -> int {
    const long long c0 = beg + (long long)i * NC;
    return (int)(end - c0 < NC ? end - c0 : NC);
  };
  // Each thread stages candidates tid (and tid + 128 when NC = 256) of every
  // chunk; records of the chunk after next are prefetched into registers
  // during the epilogue, so the gather latency hides behind the MUFU work.
  static_assert(NC <= 128, "one candidate per thread");
  float4 pre[rec_floats(N) / 4];
  if (nchunks > 0) {
    load_record<N>(a, beg, chunk_n(0), tid, pre);
    uint8_t* st = Bbuf;
    if (tid < NC)
      stage_coef<N>(pre, tid, sctr, st, st + S::B_BYTES,
                    reinterpret_cast<float*>(st + 2 * S::B_BYTES));
  }
  if (nchunks > 1) load_record<N>(a, beg + NC, chunk_n(1), tid, pre);
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
  constexpr uint32_t IDESC = idesc_tf32(NC);
  auto issue = [&](int i) {  // MMA of chunk i from stage buffer i & 1 into accumulator i & 1
    fence_after_sync();
    uint8_t* st = Bbuf + (i & 1) * STAGE;
    const uint32_t d = tmem + (uint32_t)((i & 1) * NC);
    const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo);
    const uint32_t bh = smem_u32(st), bl = smem_u32(st + S::B_BYTES);
#pragma unroll
    for (int ks = 0; ks < KP / 8; ++ks) {
      const uint32_t ko = (uint32_t)ks * 256u;  // two core matrices per K step of 8
      const uint64_t dah = smem_desc(ah + ko, 128, S::SBO_A);
      const uint64_t dal = smem_desc(al + ko, 128, S::SBO_A);
      const uint64_t dbh = smem_desc(bh + ko, 128, S::SBO_B);
      const uint64_t dbl = smem_desc(bl + ko, 128, S::SBO_B);
      mma_tf32(d, dah, dbh, IDESC, ks > 0 ? 1u : 0u);
      mma_tf32(d, dah, dbl, IDESC, 1u);
      mma_tf32(d, dal, dbh, IDESC, 1u);
    }
    mma_commit(&bar[i & 1]);
  };
  if (nchunks > 0 && tid == 0) issue(0);

  float2 acc[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  uint32_t phase[2] = {0u, 0u};
  for (int i = 0; i < nchunks; ++i) {
    // stage chunk i + 1 while the tensor core works on chunk i; its buffer
    // was last read by MMA(i - 1), which completed before epilogue(i - 1)
    if (i + 1 < nchunks && tid < NC) {
      uint8_t* st = Bbuf + ((i + 1) & 1) * STAGE;
      stage_coef<N>(pre, tid, sctr, st, st + S::B_BYTES,
                    reinterpret_cast<float*>(st + 2 * S::B_BYTES));
    }
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();  // staging done, epilogue(i - 1) done: accumulator (i + 1) & 1 is free
    if (i + 1 < nchunks && tid == 0) issue(i + 1);
    if (i + 2 < nchunks) load_record<N>(a, beg + (long long)(i + 2) * NC, chunk_n(i + 2), tid, pre);
    if (!mbar_wait_bounded(&bar[i & 1], phase[i & 1], kWaitLimit)) {
      atomicExch(&s_abort, 1);
      if (a.status) set_status(a.status, NDG_ERR_TIMEOUT);
    }
    phase[i & 1] ^= 1u;
    fence_after_sync();
    __syncthreads();  // s_abort is read only right after a barrier: uniform
    if (s_abort) break;
    const float* sw2 = reinterpret_cast<const float*>(Bbuf + (i & 1) * STAGE + 2 * S::B_BYTES);
    const uint32_t acc_addr = tmem + lane_off + (uint32_t)((i & 1) * NC);
    // all NC columns of this thread's row in flight at once, one wait
    uint32_t v[NC];
#pragma unroll
    for (int cb = 0; cb < NC; cb += 32) tmem_ld32_nowait(acc_addr + (uint32_t)cb, v + cb);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < NC; j += 2) {
      const float2 e = make_float2(ex2_approx(__uint_as_float(v[j])),
                                   ex2_approx(__uint_as_float(v[j + 1])));
      const float4 w01 = *reinterpret_cast<const float4*>(sw2 + (j >> 1) * 8);
      const float2 w2p = *reinterpret_cast<const float2*>(sw2 + (j >> 1) * 8 + 4);
      acc[0] = __ffma2_rn(make_float2(w01.x, w01.y), e, acc[0]);
      acc[1] = __ffma2_rn(make_float2(w01.z, w01.w), e, acc[1]);
      acc[2] = __ffma2_rn(w2p, e, acc[2]);
    }
    fence_before_sync();
    __syncthreads();  // the next iteration restages buffer (i + 2) & 1 = i & 1
  }
  __syncthreads();
  if (s_abort) {
    // let any MMA still in flight finish before tensor memory is released
    mbar_wait_bounded(&bar[0], phase[0], kWaitLimit);
    mbar_wait_bounded(&bar[1], phase[1], kWaitLimit);
  }
  if (active && !s_abort) {
#pragma unroll
    for (int c = 0; c < 3; ++c) a.y[(q0 + tid) * 3 + c] = acc[c].x + acc[c].y;
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tmem, S::TMEM_COLS);
  }
}

// ---- backward on the tensor cores ----------------------------------------------------
// One CTA (128 threads) per tile of up to 256 queries; thread j owns candidate
// j of a chunk of 128 (TMEM lane j).  Per chunk:
//   GEMM 1  S' = Coef Phi^T     [128 cand x 256 queries] (M = 128, N = 256,
//           K = KP features), Coef and Phi split TF32 hi/lo, 3 products;
//   pass p (32 queries each): e = 2^S', beta = e sum_c dy_c w_c,
//           sum dy e accumulated per thread; beta (hi/lo) written K-major
//           and GEMM 2 accumulates D2 += beta Phi_p  [128 cand x KP], its B
//           operand a second, transposed copy of Phi (features x queries,
//           K-major over queries: TF32 operands must be K-major);
//   dl/dcoef = -D2 / 2, chained per candidate to dl/dA, dl/dm and
//           dl/dM = 2 M G (G the symmetric gradient w.r.t. A = M^T M).
// The record [dl/dM, dl/dm, dl/dw] goes to the entry's Gaussian-major slot.
// Shared memory bounds it to N <= 6 (KP <= 32).
template <int N>
struct TcBwdShape {
  static constexpr int P = tri(N);
  static constexpr int F = P + N + 1;
  static constexpr int KP = (F + 15) / 16 * 16;  // also the N dimension of GEMM 2
  static constexpr int NC = 128, QT = 256, QB = 32;
  static constexpr uint32_t SBO_PHI = (KP / 4) * 128;
  static constexpr uint32_t PHI_BYTES = (uint32_t)QT * KP * 4;
  static constexpr uint32_t SBO_PT = (QT / 4) * 128;  // transposed copy: 8-feature groups
  static constexpr uint32_t PT_BYTES = (uint32_t)KP * QT * 4;
  static constexpr uint32_t SBO_C = (KP / 4) * 128;
  static constexpr uint32_t C_BYTES = (uint32_t)NC * KP * 4;
  static constexpr uint32_t SBO_BETA = (QB / 4) * 128;
  static constexpr uint32_t BETA_BYTES = (uint32_t)NC * QB * 4;
  static constexpr uint32_t SMEM_USED =
      2 * PHI_BYTES + 2 * PT_BYTES + 2 * C_BYTES + 2 * BETA_BYTES + QT * 16 + 128;
  // one CTA per SM: the kernel allocates all 512 tensor-memory columns
  static constexpr uint32_t SMEM = SMEM_USED > 117u * 1024u ? SMEM_USED : 117u * 1024u;
  static_assert(SMEM <= 227u * 1024u, "shared memory");
};

template <int N>
__global__ void __launch_bounds__(128, 1) bwd_tc_kernel(BwdArgs a) {
  using S = TcBwdShape<N>;
  constexpr int P = S::P, KP = S::KP, NC = S::NC, QB = S::QB, R = rec_floats(N), R4 = R / 4;
  constexpr int RP = part_floats(N);
  extern __shared__ __align__(128) uint8_t dsm[];
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm + 127) & ~(uintptr_t)127);
  uint8_t* Phh = base;
  uint8_t* Phl = Phh + S::PHI_BYTES;
  uint8_t* Pth = Phl + S::PHI_BYTES;
  uint8_t* Ptl = Pth + S::PT_BYTES;
  uint8_t* Ch = Ptl + S::PT_BYTES;
  uint8_t* Cl = Ch + S::C_BYTES;
  uint8_t* Bh = Cl + S::C_BYTES;
  uint8_t* Bl = Bh + S::BETA_BYTES;
  float4* sdy = reinterpret_cast<float4*>(Bl + S::BETA_BYTES);
  __shared__ uint64_t bar1, bar2;
  __shared__ uint32_t tmem_base;
  __shared__ float sred[4 * N * 2];
  __shared__ float sctr[N];
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5;
  const long long t = blockIdx.x;
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
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int qi = tid + 128 * h;
      const bool v = qi < nq;
      float xt[N];
#pragma unroll
      for (int d = 0; d < N; ++d) xt[d] = v ? (h ? xb[d] : xa[d]) - sctr[d] : 0.0f;
      float phi[KP];
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) phi[tri(i) + j] = xt[i] * xt[j];
#pragma unroll
      for (int i = 0; i < N; ++i) phi[P + i] = xt[i];
      phi[P + N] = v ? 1.0f : 0.0f;
#pragma unroll
      for (int k = P + N + 1; k < KP; ++k) phi[k] = 0.0f;
      store_row_split<KP>(Phh, Phl, qi, S::SBO_PHI, phi);
      // transposed copy: element (f, qi), K-major over queries
#pragma unroll
      for (int f = 0; f < KP; ++f) {
        const float hv = tf32_hi(phi[f]);
        const uint32_t off = kmajor_off(f, qi, S::SBO_PT);
        *reinterpret_cast<float*>(Pth + off) = hv;
        *reinterpret_cast<float*>(Ptl + off) = phi[f] - hv;
      }
      sdy[qi] = v ? make_float4(a.dy[(q0 + qi) * 3], a.dy[(q0 + qi) * 3 + 1],
                                a.dy[(q0 + qi) * 3 + 2], 0.0f)
                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar1, 1);
    mbar_init(&bar2, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t d2_col = 256;
  constexpr uint32_t IDESC1 = idesc_tf32(256);
  constexpr uint32_t IDESC2 = idesc_tf32(KP);
  const int npass = (nq + QB - 1) / QB;
  uint32_t ph1 = 0, ph2 = 0;
  const long long beg = a.offsets[t], end = a.offsets[t + 1];
  for (long long c0 = beg; c0 < end; c0 += NC) {
    const int n = (int)(end - c0 < NC ? end - c0 : NC);
    // ---- stage candidate tid: record, A = M^T M, coefficients
    const int g = tid < n ? a.ids[c0 + tid] : -1;
    const bool live = (unsigned)g < (unsigned)a.Ge;
    float M[P], mt[N], w[3];
    {
      float buf[R];
      if (live) {
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
      for (int i = 0; i < P; ++i) M[i] = buf[i];
#pragma unroll
      for (int i = 0; i < N; ++i) mt[i] = live ? buf[P + i] - sctr[i] : 0.0f;
#pragma unroll
      for (int c = 0; c < 3; ++c) w[c] = buf[P + N + c];
    }
    float A[P];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) {
        float s2 = 0.0f;
#pragma unroll
        for (int k = i; k < N; ++k) s2 = fmaf(M[tri(k) + i], M[tri(k) + j], s2);
        A[tri(i) + j] = s2;
      }
    {
      float coef[KP];
      float u[N], cst = 0.0f;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float s2 = 0.0f;
#pragma unroll
        for (int k = 0; k < N; ++k) s2 = fmaf(A[i >= k ? tri(i) + k : tri(k) + i], mt[k], s2);
        u[i] = s2;
        cst = fmaf(mt[i], s2, cst);
      }
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int k = 0; k <= i; ++k)
          coef[tri(i) + k] = kNegHalfLog2eTC * (i == k ? A[tri(i) + k] : 2.0f * A[tri(i) + k]);
#pragma unroll
      for (int i = 0; i < N; ++i) coef[P + i] = kNegHalfLog2eTC * (-2.0f * u[i]);
      coef[P + N] = kNegHalfLog2eTC * cst;
#pragma unroll
      for (int k = P + N + 1; k < KP; ++k) coef[k] = 0.0f;
      store_row_split<KP>(Ch, Cl, tid, S::SBO_C, coef);
    }
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint32_t ch = smem_u32(Ch), cl = smem_u32(Cl), ph = smem_u32(Phh), pl = smem_u32(Phl);
#pragma unroll
      for (int ks = 0; ks < KP / 8; ++ks) {
        const uint32_t ko = (uint32_t)ks * 256u;
        const uint64_t dch = smem_desc(ch + ko, 128, S::SBO_C);
        const uint64_t dcl = smem_desc(cl + ko, 128, S::SBO_C);
        const uint64_t dph = smem_desc(ph + ko, 128, S::SBO_PHI);
        const uint64_t dpl = smem_desc(pl + ko, 128, S::SBO_PHI);
        mma_tf32(tmem, dch, dph, IDESC1, ks > 0 ? 1u : 0u);
        mma_tf32(tmem, dch, dpl, IDESC1, 1u);
        mma_tf32(tmem, dcl, dph, IDESC1, 1u);
      }
      mma_commit(&bar1);
    }
    if (!mbar_wait_bounded(&bar1, ph1, kWaitLimit)) {
      atomicExch(&s_abort, 1);
      if (a.status) set_status(a.status, NDG_ERR_TIMEOUT);
    }
    ph1 ^= 1u;
    fence_after_sync();
    __syncthreads();  // s_abort is read only right after a barrier: uniform
    if (s_abort) break;
    float Gw[3] = {0.f, 0.f, 0.f};
    for (int p = 0; p < npass; ++p) {
      if (p > 0) {  // beta is still being read by the previous pass's GEMM 2
        if (!mbar_wait_bounded(&bar2, ph2, kWaitLimit)) {
          atomicExch(&s_abort, 1);
          if (a.status) set_status(a.status, NDG_ERR_TIMEOUT);
        }
        ph2 ^= 1u;
        fence_after_sync();
        __syncthreads();
        if (s_abort) break;
      }
#pragma unroll 1
      for (int cb = 0; cb < QB; cb += 32) {
        float v[32];
        tmem_ld32(lane_addr + (uint32_t)(p * QB + cb), v);
#pragma unroll
        for (int q4 = 0; q4 < 32; q4 += 4) {
          float bh[4], bl[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float e = ex2_approx(v[q4 + r]);
            const float4 dq = sdy[p * QB + cb + q4 + r];
            const float wd = fmaf(dq.x, w[0], fmaf(dq.y, w[1], dq.z * w[2]));
            const float beta = e * wd;
            Gw[0] = fmaf(dq.x, e, Gw[0]);
            Gw[1] = fmaf(dq.y, e, Gw[1]);
            Gw[2] = fmaf(dq.z, e, Gw[2]);
            bh[r] = tf32_hi(beta);
            bl[r] = beta - bh[r];
          }
          const uint32_t off = kmajor_off(tid, cb + q4, S::SBO_BETA);
          *reinterpret_cast<float4*>(Bh + off) = make_float4(bh[0], bh[1], bh[2], bh[3]);
          *reinterpret_cast<float4*>(Bl + off) = make_float4(bl[0], bl[1], bl[2], bl[3]);
        }
      }
      fence_proxy_async();
      fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        fence_after_sync();
        const uint32_t bh = smem_u32(Bh), bl = smem_u32(Bl), ph = smem_u32(Pth), pl = smem_u32(Ptl);
#pragma unroll
        for (int ks = 0; ks < QB / 8; ++ks) {
          // queries p QB + 8 ks .. + 8: two 4-query core columns of Phi^T
          const uint32_t ko = (uint32_t)(p * QB / 4 + 2 * ks) * 128u;
          const uint64_t dbh = smem_desc(bh + (uint32_t)ks * 256u, 128, S::SBO_BETA);
          const uint64_t dbl = smem_desc(bl + (uint32_t)ks * 256u, 128, S::SBO_BETA);
          const uint64_t dph = smem_desc(ph + ko, 128, S::SBO_PT);
          const uint64_t dpl = smem_desc(pl + ko, 128, S::SBO_PT);
          mma_tf32(tmem + d2_col, dbh, dph, IDESC2, (p > 0 || ks > 0) ? 1u : 0u);
          mma_tf32(tmem + d2_col, dbh, dpl, IDESC2, 1u);
          mma_tf32(tmem + d2_col, dbl, dph, IDESC2, 1u);
        }
        mma_commit(&bar2);
      }
    }
    __syncthreads();
    if (s_abort) break;
    if (npass > 0) {
      if (!mbar_wait_bounded(&bar2, ph2, kWaitLimit)) {
        atomicExch(&s_abort, 1);
        if (a.status) set_status(a.status, NDG_ERR_TIMEOUT);
      }
      ph2 ^= 1u;
      fence_after_sync();
    }
    __syncthreads();
    if (s_abort) break;
    // ---- epilogue 2: dl/dcoef -> record
    float Gc[KP];
#pragma unroll
    for (int cb = 0; cb < KP; cb += 16) {
      float v[16];
      tmem_ld16(lane_addr + d2_col + (uint32_t)cb, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) Gc[cb + i] = -0.5f * v[i];
    }
    if (tid < n && live) {
      const float Gc0 = Gc[P + N];
      // symmetric gradient w.r.t. A (full matrix entries), from the
      // coefficients [A_ii | 2 A_ij, -2 A m~, m~^T A m~]
      float Gf[N][N];
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int k = 0; k <= i; ++k) {
          float gv;
          if (i == k) {
            gv = Gc[tri(i) + i] - 2.0f * Gc[P + i] * mt[i] + Gc0 * mt[i] * mt[i];
          } else {
            gv = Gc[tri(i) + k] - (Gc[P + i] * mt[k] + Gc[P + k] * mt[i]) + Gc0 * mt[i] * mt[k];
          }
          Gf[i][k] = gv;
          Gf[k][i] = gv;
        }
      float rec[RP];
      // dl/dM = 2 M G (lower part): (M G)_ik = sum_{l <= i} M_il G_lk
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int k = 0; k <= i; ++k) {
          float s2 = 0.0f;
#pragma unroll
          for (int l = 0; l <= i; ++l) s2 = fmaf(M[tri(i) + l], Gf[l][k], s2);
          rec[tri(i) + k] = 2.0f * s2;
        }
      // dl/dm = dl/dm~ = 2 A (Gc0 m~ - G_lin)
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float s2 = 0.0f;
#pragma unroll
        for (int k = 0; k < N; ++k)
          s2 = fmaf(A[i >= k ? tri(i) + k : tri(k) + i], Gc0 * mt[k] - Gc[P + k], s2);
        rec[P + i] = 2.0f * s2;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) rec[P + N + c] = Gw[c];
#pragma unroll
      for (int i = P + N + 3; i < RP; ++i) rec[i] = 0.0f;
      const long long slot = a.slot ? (long long)a.slot[c0 + tid] : c0 + tid;
      float* out = a.part + (size_t)slot * RP;
#pragma unroll
      for (int i = 0; i < RP; i += 4)
        *reinterpret_cast<float4*>(out + i) = make_float4(rec[i], rec[i + 1], rec[i + 2], rec[i + 3]);
    }
    fence_before_sync();
    __syncthreads();
  }
  if (s_abort) {
    mbar_wait_bounded(&bar1, ph1, kWaitLimit);
    mbar_wait_bounded(&bar2, ph2, kWaitLimit);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tmem, 512);
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

int launch_fwd_tc(int N, const FwdArgs& a, long long T, cudaStream_t s) {
  if (T <= 0) return 0;
  if (N <= 8) return launch_fwd_h(N, a, T, s);  // FP16-split kernel
  const long long blocks = T * ((a.tile + 127) / 128);
#define L_TC(n)                                                                              \
  {                                                                                          \
    cudaFuncSetAttribute(fwd_tc_kernel<n>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                         (int)TcShape<n>::SMEM);                                             \
    fwd_tc_kernel<n><<<(unsigned)blocks, 128, TcShape<n>::SMEM, s>>>(a);                     \
  }
  switch (N) {
    NDG_CASE_N(9, L_TC) NDG_CASE_N(10, L_TC) NDG_CASE_N(11, L_TC) NDG_CASE_N(12, L_TC)
    default: return 0;
  }
#undef L_TC
  return 1;
}

int launch_bwd_tc(int N, const BwdArgs& a, long long T, cudaStream_t s) {
  if (T <= 0) return 0;
#define L_BTC(n)                                                                             \
  {                                                                                          \
    cudaFuncSetAttribute(bwd_tc_kernel<n>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                         (int)TcBwdShape<n>::SMEM);                                          \
    bwd_tc_kernel<n><<<(unsigned)T, 128, TcBwdShape<n>::SMEM, s>>>(a);                       \
  }
  switch (N) {
    NDG_CASE_N(1, L_BTC) NDG_CASE_N(2, L_BTC) NDG_CASE_N(3, L_BTC) NDG_CASE_N(4, L_BTC)
    NDG_CASE_N(5, L_BTC) NDG_CASE_N(6, L_BTC)
    default: return 0;
  }
#undef L_BTC
  return 1;
}

size_t fwd_tc_smem(int N) {
  size_t v = 0;
#define L_SZ(n) v = TcShape<n>::SMEM
  NDG_SWITCH_N(N, L_SZ)
#undef L_SZ
  return v;
}

}  // namespace ndg
