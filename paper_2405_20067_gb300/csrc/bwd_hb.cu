// bwd_hb.cu -- the analytic backward on the tensor cores in the beta form
// (ndg_backward, NDG_MODE_TC, N = 7..12; built for every N <= 12, while
// N <= 6 dispatches the E Psi form of bwd_h.cu, measured faster there).
//
// With the lifted form of the forward (s = phi(x~) . coef, e = 2^s, the
// coefficients scaled by -log2(e) / 2), the gradients of an entry (Gaussian
// j, tile) are sums over the tile's queries q:
//   dl/dc_k  = -1/2 sum_q beta_jq phi_qk,   beta_jq = e_jq sum_c dy_qc w_jc
//   dl/dw_jc = sum_q e_jq dy_qc
// (dl/dc: the lifted coefficients; beta: the pair's weight in the exponent's
// gradient).  Per chunk of 128 candidates and unit of 128 queries:
//   MMA 1    S^T = Coef Phi^T (candidates on the TMEM lanes), FP16 hi / lo
//            operands, three products (the exponent needs ~22 bits);
//   epilogue e = 2^S; beta' = e (dy'_q . w_j) written back in place as FP16
//            (the A operand of MMA 2); sum_q e dy'_qc accumulated in FP32;
//   MMA 2    D = beta' Phi (K = the unit's queries).  Phi is stored once per
//            tile with the hi and the lo parts of each 8-query group side by
//            side: MMA 1 reads it K-major (queries on N), MMA 2 MN-major
//            (features on N), so that one MMA's N spans the hi and the lo
//            features (2 KP) where that fits tensor memory (N <= 9), else
//            hi and lo are two MMAs of N = KP accumulating into one block.
// Precision: phi keeps hi + lo (the record's cancellation amplifies its
// rounding), dl/dw stays FP32, and beta' is rounded once to FP16 after a
// per-candidate power-of-two scale 1/rho that brings the largest weight into
// (1/2, 1]: unscaled, a dim Gaussian's beta' (a child starts near weight
// 1e-3) falls among the FP16 subnormals, which cost 1e-3 relative in the
// children's gradients at N = 12.  Measured 1e-4 to 6e-4 relative per
// gradient tensor for N = 1..12; an FP16 lo part of beta' (a third product)
// gained less than 1.5x at N = 12 for 10% more time at N = 10.
//
// Per entry the chain (epilogue warps, one chunk behind) turns D into the
// frame-free record [G = dl/dA (symmetric, lower packed), v = Gc0 m~ - G_lin,
// dl/dw] (dl/dM = 2 M sum G and dl/dm = 2 A sum v follow per Gaussian after
// the segmented sum), written in entry order.
//
// CTA = one tile of up to 256 queries, 416 threads, one CTA per SM:
//   warps 0-3   builders: coefficient rows of chunk i into coefficient stage
//               i % CS, the chunk's per-candidate data (m~, w / rho, entry,
//               row factor, rho) into stash slot i % SS;
//   warp 12     MMA issuer (lane 0): MMA 1 of unit u + LEAD, then MMA 2 of u;
//   warps 4-11  epilogue: warp w owns TMEM lanes 32 (w % 4) .. + 31 (its
//               candidates) and 64 columns (queries) of each unit; after the
//               last unit of chunk i it forms half of the record parts of
//               chunk i - 1 (the builders held the next chunk's records in
//               registers, and the chain there spilled).
// TMEM: NBUF S buffers of 128 columns, then two D buffers.  Every wait is
// bounded; a timeout records NDG_ERR_TIMEOUT and the CTA lets its issued
// MMAs finish (bounded) before it frees tensor memory.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "kernels.h"
#include "tcgen05.cuh"

namespace ndg {

template <int N>
struct BwdBShape {
  static constexpr int P = tri(N);
  static constexpr int F = P + N + 1;
  static constexpr int KP = (F + 15) / 16 * 16;
  static constexpr int NC = 128;  // candidates per chunk (MMA 1 M, TMEM lanes)
  static constexpr int UQ = 128;  // queries per unit (MMA 1 N, MMA 2 K)
  // MMA 2 over hi and lo together (N = 2 KP) when two such D buffers and two
  // S buffers fit the 512 columns
  static constexpr bool MERGE = 4 * KP + 256 <= 512;
  static constexpr int ND = MERGE ? 2 * KP : KP;  // D columns per buffer
  static constexpr int NBUF = (512 - 2 * ND) / 128 >= 3 ? 3 : 2;
  static constexpr uint32_t TM_D = NBUF * 128;
  static constexpr int R = rec_floats(N);
  static constexpr int R2 = rec_tc_floats(N);
  static constexpr int RPT = part_floats(N);  // per-entry record floats
  static constexpr int RQT = RPT / 4;
  static constexpr int NPART = N <= 8 ? 2 : 4;  // the record is formed in parts
  static constexpr int PARTW = (RPT / NPART + 3) / 4 * 4;
  static constexpr int PQMAX = PARTW / 4;
  // staging row stride in float4s: odd, so that 8 consecutive rows' 16-byte
  // stores fall in distinct banks
  static constexpr int PQS = PQMAX | 1;
  // Phi: per 8-query group, hi cores (KP / 8 x 128 B) then lo cores
  static constexpr uint32_t GRP = 2u * KP * 16;         // bytes per 8-query group
  static constexpr uint32_t LO_OFF = (uint32_t)KP * 16;  // lo cores inside a group
  static constexpr uint32_t PHI_BYTES = 32u * GRP;       // 256 queries
  static constexpr uint32_t SBO_C = (KP / 8) * 128;      // coefficient rows: 8-row groups
  static constexpr uint32_t C_BYTES = (uint32_t)NC * KP * 2;
  static constexpr uint32_t C_STAGE = 2 * C_BYTES;       // hi, lo
  // stash slot: SV fields per candidate, field-major ([SV][NC]: lane j
  // reads word j of a field, conflict-free): m~ (N), w / rho (3), entry,
  // row factor, rho; then the two column halves' sum_q e dy' (float4 each)
  static constexpr int SV = (N + 6 + 3) / 4 * 4;
  static constexpr uint32_t SLOT = (uint32_t)NC * SV * 4 + 2u * NC * 16;
  static constexpr int SS = N >= 9 ? 3 : 4;  // >= 3: the chain runs one chunk behind the epilogue
  static constexpr uint32_t DYC = 3u * 256 * 4;  // dy' by colour
  static constexpr uint32_t OUT_BYTES = 16u * PQS * 16;
  static constexpr uint32_t FIXED = PHI_BYTES + SS * SLOT + DYC + 8 * OUT_BYTES + 128 + 4096;
  // coefficient stages: as many as fit (up to 3; N = 12 has room for one)
  static constexpr int CS = FIXED + 3 * C_STAGE <= 227u * 1024u   ? 3
                            : FIXED + 2 * C_STAGE <= 227u * 1024u ? 2
                                                                  : 1;
  static constexpr uint32_t SMEM_USED = FIXED - 4096 + CS * C_STAGE;
  static constexpr uint32_t SMEM = SMEM_USED > 116u * 1024u ? SMEM_USED : 116u * 1024u;
  static_assert(TM_D + 2 * ND <= 512, "tensor memory");
  static_assert(FIXED + CS * C_STAGE <= 227u * 1024u, "shared memory");
  static_assert(ND % 16 == 0 && ND <= 256, "MMA 2 shape");
  static_assert(NPART * PARTW >= RPT, "record parts");
};

namespace {

__device__ __forceinline__ void split_hb(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(v0, v1);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(v0 - hf.x, v1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// byte offset of element (row, k) of a K-major no-swizzle FP16 operand whose
// 8-row groups are sbo bytes apart
__device__ __forceinline__ uint32_t coff(int row, int k, uint32_t sbo) {
  return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k & 7) * 2u;
}

constexpr float kNegHalfLog2eBB = -0.72134752044448170368f;
constexpr float kRowMaxC = 16384.0f;

// Which lifted-coefficient gradients Gc_k the record positions [p0, p1) use:
// G(d, e) needs Gc_de, Gc_lin_d, Gc_lin_e and Gc0; v_i needs Gc_lin_i and
// Gc0; dl/dw needs none.  As two 64-bit words (F <= 91): word wd holds
// k = 64 wd .. 64 wd + 63.
__host__ __device__ constexpr bool kneed(unsigned long long w0, unsigned long long w1, int k) {
  return (((k >> 6) ? w1 : w0) >> (k & 63)) & 1ull;
}
template <int N>
__host__ __device__ constexpr unsigned long long chain_mask_word(int p0, int p1, int wd) {
  unsigned long long m = 0ull;
  constexpr int P = tri(N);
  for (int d = 0; d < N; ++d)
    for (int e = 0; e <= d; ++e) {
      const int p = tri(d) + e;
      if (p >= p0 && p < p1) {
        const int ks[4] = {p, P + d, P + e, P + N};
        for (int q = 0; q < 4; ++q)
          if ((ks[q] >> 6) == wd) m |= 1ull << (ks[q] & 63);
      }
    }
  for (int i = 0; i < N; ++i)
    if (P + i >= p0 && P + i < p1) {
      const int ks[2] = {P + i, P + N};
      for (int q = 0; q < 2; ++q)
        if ((ks[q] >> 6) == wd) m |= 1ull << (ks[q] & 63);
    }
  return m;
}

}  // namespace

template <int N>
__global__ void __launch_bounds__(416, 1) bwd_hb_kernel(BwdArgs a) {
  using S = BwdBShape<N>;
  constexpr int P = S::P, F = S::F, KP = S::KP, NC = S::NC, CS = S::CS, SS = S::SS;
  constexpr int R4 = S::R / 4, R2 = S::R2, SV = S::SV, NBUF = S::NBUF, ND = S::ND;
  extern __shared__ __align__(128) uint8_t dsm[];
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm + 127) & ~(uintptr_t)127);
  uint8_t* Phi = base;
  uint8_t* Cst = Phi + S::PHI_BYTES;                   // CS coefficient stages (hi, lo)
  uint8_t* Slots = Cst + CS * S::C_STAGE;              // SS stash slots
  float* sdyc = reinterpret_cast<float*>(Slots + SS * S::SLOT);  // dy' [3][256]
  float4* Outs = reinterpret_cast<float4*>(sdyc + 3 * 256);       // 8 x OUT_BYTES
  __shared__ uint64_t coef_full[CS], coef_empty[CS], stash_full[SS], stash_empty[SS], gw_full[SS],
      s_full[NBUF], e_full[NBUF], d_full[2], d_empty[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ float sred[8 * N * 2], sdy[8];
  __shared__ float sctr[N], sh[N], s_dys;
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long t = blockIdx.x;
  const long long qt = t * a.tile;
  const int nq = (int)(a.Q - qt < a.tile ? a.Q - qt : a.tile);
  const int nh = (nq + S::UQ - 1) / S::UQ;  // units per chunk

  if (tid == 0) {
    for (int i = 0; i < CS; ++i) {
      mbar_init(&coef_full[i], 4);
      mbar_init(&coef_empty[i], 1);  // MMA 1 (commit)
    }
    for (int i = 0; i < SS; ++i) {
      mbar_init(&stash_full[i], 4);
      mbar_init(&stash_empty[i], 8);  // the chain
      mbar_init(&gw_full[i], 8);      // the epilogue's sum_q e dy'
    }
    for (int i = 0; i < NBUF; ++i) {
      mbar_init(&s_full[i], 1);
      mbar_init(&e_full[i], 8);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&d_full[i], 1);
      mbar_init(&d_empty[i], 8);
    }
    mbar_init(&drain, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  // ---- per tile: centre, feature and dy scales, Phi rows and dy'
  const bool is_epi = warp >= 4 && warp < 12;
  const int row = tid - 128;
  const bool active_row = is_epi && row < nq;
  float xq[N], dq[3];
#pragma unroll
  for (int d = 0; d < N; ++d) xq[d] = active_row ? a.x[(qt + row) * N + d] : 0.0f;
#pragma unroll
  for (int c = 0; c < 3; ++c) dq[c] = active_row ? a.dy[(qt + row) * 3 + c] : 0.0f;
  if (is_epi) {
#pragma unroll
    for (int d = 0; d < N; ++d) {
      float lo = active_row ? xq[d] : INFINITY, hi = active_row ? xq[d] : -INFINITY;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      if (lane == 0) {
        sred[((warp - 4) * N + d) * 2] = lo;
        sred[((warp - 4) * N + d) * 2 + 1] = hi;
      }
    }
    float m = fmaxf(fmaxf(fabsf(dq[0]), fabsf(dq[1])), fabsf(dq[2]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) sdy[warp - 4] = m;
  }
  __syncthreads();
  if (tid < N) {
    float lo = INFINITY, hi = -INFINITY;
    for (int w = 0; w < 8; ++w) {
      lo = fminf(lo, sred[(w * N + tid) * 2]);
      hi = fmaxf(hi, sred[(w * N + tid) * 2 + 1]);
    }
    const float c = (lo <= hi) ? 0.5f * (lo + hi) : 0.0f;
    sctr[tid] = c;
    sh[tid] = (lo <= hi) ? pow2_ceil(fmaxf(hi - c, c - lo)) : 1.0f;
  }
  if (tid == N) {
    float m = 0.0f;
    for (int w = 0; w < 8; ++w) m = fmaxf(m, sdy[w]);
    s_dys = pow2_ceil(m);
  }
  __syncthreads();
  if (is_epi) {
    float u[N];
#pragma unroll
    for (int d = 0; d < N; ++d) u[d] = active_row ? (xq[d] - sctr[d]) * (1.0f / sh[d]) : 0.0f;
    float phi[KP];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) phi[tri(i) + j] = u[i] * u[j];
#pragma unroll
    for (int i = 0; i < N; ++i) phi[P + i] = u[i];
    phi[P + N] = active_row ? 1.0f : 0.0f;
#pragma unroll
    for (int k = F; k < KP; ++k) phi[k] = 0.0f;
    // row `row` of Phi: hi cores, then lo cores, of its 8-query group
#pragma unroll
    for (int k = 0; k < KP; k += 8) {
      uint4 h, l;
      split_hb(phi[k], phi[k + 1], h.x, l.x);
      split_hb(phi[k + 2], phi[k + 3], h.y, l.y);
      split_hb(phi[k + 4], phi[k + 5], h.z, l.z);
      split_hb(phi[k + 6], phi[k + 7], h.w, l.w);
      const uint32_t off = coff(row, k, S::GRP);
      *reinterpret_cast<uint4*>(Phi + off) = h;
      *reinterpret_cast<uint4*>(Phi + S::LO_OFF + off) = l;
    }
    const float idys = 1.0f / s_dys;
#pragma unroll
    for (int c = 0; c < 3; ++c) sdyc[c * 256 + row] = dq[c] * idys;  // zero past the tile
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  const long long beg = a.offsets[t], end = a.offsets[t + 1];
  const int nchunks = (int)((end - beg + NC - 1) / NC);
  const int U = nchunks * nh;
  volatile int* abort_flag = &s_abort;
  auto fail = [&]() {
    atomicExch(&s_abort, 1);
    if (a.status) set_status(a.status, NDG_ERR_TIMEOUT);
  };
  auto slot_f = [&](int i) -> float* { return reinterpret_cast<float*>(Slots + (i % SS) * S::SLOT); };

  if (warp < 4) {
    // ---- builders (thread j = candidate j of each chunk)
    const int j = tid;
    float hsc[N];
#pragma unroll
    for (int d = 0; d < N; ++d) hsc[d] = sh[d];
    auto cand = [&](int i) -> int2 {
      const long long e = beg + (long long)i * NC + j;
      const bool in = i < nchunks && e < end;
      const int g = in ? a.ids[e] : -1;
      const bool live = (unsigned)g < (unsigned)a.Ge;
      return make_int2(live ? g : -1, live ? (int)e : -1);
    };
    auto load = [&](int g, float4 (&r)[R4]) {
      if (g >= 0) {
        const float4* src = reinterpret_cast<const float4*>(a.rec + (size_t)g * R2);
#pragma unroll
        for (int k = 0; k < R4; ++k) r[k] = __ldg(src + k);
      } else {
#pragma unroll
        for (int k = 0; k < R4; ++k) r[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    auto build = [&](int i, const float4 (&cur)[R4], int slot) -> bool {
      const int s = i % CS;
      if (i >= CS && !warp_wait(&coef_empty[s], ((i / CS) - 1) & 1, abort_flag)) return false;
      if (i >= SS && !warp_wait(&stash_empty[i % SS], ((i / SS) - 1) & 1, abort_flag)) return false;
      float buf[S::R];
#pragma unroll
      for (int k = 0; k < R4; ++k) {
        buf[4 * k] = cur[k].x; buf[4 * k + 1] = cur[k].y;
        buf[4 * k + 2] = cur[k].z; buf[4 * k + 3] = cur[k].w;
      }
      float coef[KP], mt[N];
#pragma unroll
      for (int d = 0; d < N; ++d) mt[d] = buf[P + d] - sctr[d];
      float cst = 0.0f;
#pragma unroll
      for (int d = 0; d < N; ++d) {
        float s2 = 0.0f;
#pragma unroll
        for (int k = 0; k < N; ++k) s2 = fmaf(buf[d >= k ? tri(d) + k : tri(k) + d], mt[k], s2);
        coef[P + d] = (kNegHalfLog2eBB * -2.0f) * s2 * hsc[d];
        cst = fmaf(mt[d], s2, cst);
      }
#pragma unroll
      for (int d = 0; d < N; ++d)
#pragma unroll
        for (int k = 0; k <= d; ++k)
          coef[tri(d) + k] = kNegHalfLog2eBB * (d == k ? buf[tri(d) + k] : 2.0f * buf[tri(d) + k]) *
                             (hsc[d] * hsc[k]);
      coef[P + N] = kNegHalfLog2eBB * cst;
#pragma unroll
      for (int k = F; k < KP; ++k) coef[k] = 0.0f;
      float mx = 0.0f;
#pragma unroll
      for (int k = 0; k < F; ++k) mx = fmaxf(mx, fabsf(coef[k]));
      float back = 1.0f;
      if (mx > kRowMaxC) {
        int ex = (int)((__float_as_uint(mx) >> 23) & 0xffu) - 127 - 13;
        ex = ex > 120 ? 120 : ex;
        const float down = __uint_as_float((uint32_t)(127 - ex) << 23);
        back = __uint_as_float((uint32_t)(127 + ex) << 23);
#pragma unroll
        for (int k = 0; k < KP; ++k) coef[k] *= down;
      }
      uint8_t* st = Cst + s * S::C_STAGE;
#pragma unroll
      for (int k = 0; k < KP; k += 8) {
        uint4 h, l;
        split_hb(coef[k], coef[k + 1], h.x, l.x);
        split_hb(coef[k + 2], coef[k + 3], h.y, l.y);
        split_hb(coef[k + 4], coef[k + 5], h.z, l.z);
        split_hb(coef[k + 6], coef[k + 7], h.w, l.w);
        const uint32_t off = coff(j, k, S::SBO_C);
        *reinterpret_cast<uint4*>(st + off) = h;
        *reinterpret_cast<uint4*>(st + S::C_BYTES + off) = l;
      }
      fence_proxy_async();
      warp_arrive(&coef_full[s]);
      // stash: m~, w / rho, entry, row factor, rho (read by the epilogue and
      // the chain).  rho, a power of two, brings the largest weight into
      // (1/2, 1], so that beta' = e (dy' . w / rho) stays clear of the FP16
      // subnormals for dim Gaussians (a child starts near 1e-3); the chain
      // scales the D row back by rho, exactly.
      const float wm = fmaxf(fmaxf(fabsf(buf[P + N]), fabsf(buf[P + N + 1])), fabsf(buf[P + N + 2]));
      const uint32_t wexp = (__float_as_uint(wm) >> 23) & 0xffu;
      const float rho = (wexp >= 1u && wexp <= 253u) ? __uint_as_float((wexp + 1u) << 23) : 1.0f;
      const float irho = 1.0f / rho;  // exact: a power of two
      float sv[N + 6];
#pragma unroll
      for (int d = 0; d < N; ++d) sv[d] = mt[d];
#pragma unroll
      for (int c = 0; c < 3; ++c) sv[N + c] = buf[P + N + c] * irho;
      sv[N + 3] = __int_as_float(slot);
      sv[N + 4] = back;
      sv[N + 5] = rho;
      float* dst = slot_f(i) + j;
#pragma unroll
      for (int k = 0; k < N + 6; ++k) dst[k * NC] = sv[k];
      warp_arrive(&stash_full[i % SS]);
      return true;
    };
    // records: N <= 6 loads chunk i + 1 while chunk i is built; larger records
    // load after the build (register budget)
    constexpr bool PRE = N <= 6;
    float4 cur[R4], nxt[PRE ? R4 : 1];
    int2 ci = cand(0);
    load(ci.x, cur);
    int slot_cur = ci.y;
    int2 c_next = cand(1);
    bool ok = true;
    for (int i = 0; i < nchunks; ++i) {
      int slot_nxt = c_next.y;
      if constexpr (PRE) {
        load(c_next.x, nxt);
        c_next = cand(i + 2);
      }
      ok = build(i, cur, slot_cur);
      if constexpr (PRE) {
#pragma unroll
        for (int k = 0; k < R4; ++k) cur[k] = nxt[k];
      } else {
        load(c_next.x, cur);
        c_next = cand(i + 2);
      }
      slot_cur = slot_nxt;
      if (__shfl_sync(0xffffffffu, (!ok || *abort_flag) ? 1 : 0, 0)) {
        ok = false;
        break;
      }
    }
    if (!ok && lane == 0) fail();
  } else if (warp == 12) {
    // ---- MMA issuer
    if (lane == 0 && U > 0) {
      constexpr uint32_t IDESC1 = idesc_f16(S::UQ);
      // MMA 2: B = Phi read MN-major (features on N); instruction bit 16
      constexpr uint32_t IDESC2 = idesc_f16(ND) | (1u << 16);
      // descriptor bases (a descriptor for base + off is base + off / 16)
      const uint64_t dPhiK = smem_desc(smem_u32(Phi), 128, S::GRP);  // K-major: queries on N
      // MN-major (features on N): the leading byte offset is the stride of the
      // 8-query groups along K, the stride byte offset that of the 8-feature
      // cores along N (checked numerically on GB300)
      const uint64_t dPhiM = smem_desc(smem_u32(Phi), S::GRP, 128);
      const uint64_t dC0 = smem_desc(smem_u32(Cst), 128, S::SBO_C);
      constexpr uint64_t PHI_LO = S::LO_OFF >> 4, C_LO = S::C_BYTES >> 4;
      auto mma1 = [&](int u) -> bool {
        const int i = u / nh, h = u - i * nh, s = i % CS, sb = u % NBUF;
        if (h == 0 && !mbar_wait_sleep(&coef_full[s], (i / CS) & 1, abort_flag)) return false;
        fence_after_sync();
        const uint64_t dch = dC0 + (uint64_t)((s * S::C_STAGE) >> 4);
        const uint64_t dph = dPhiK + (uint64_t)((h * 16 * S::GRP) >> 4);  // 16 groups per unit
        const uint32_t d = tmem + (uint32_t)(sb * S::UQ);
#pragma unroll
        for (int ks = 0; ks < KP / 16; ++ks) {
          const uint64_t ko = (uint64_t)ks * 16u;  // two 128-byte cores per K step
          mma_f16(d, dch + ko, dph + ko, IDESC1, ks > 0 ? 1u : 0u);
          mma_f16(d, dch + ko, dph + PHI_LO + ko, IDESC1, 1u);
          mma_f16(d, dch + C_LO + ko, dph + ko, IDESC1, 1u);
        }
        mma_commit(&s_full[sb]);
        if (h == nh - 1) mma_commit(&coef_empty[s]);
        return true;
      };
      auto mma2 = [&](int u) -> bool {
        const int i = u / nh, h = u - i * nh, sb = u % NBUF, db = i & 1;
        if (!mbar_wait_sleep(&e_full[sb], (u / NBUF) & 1, abort_flag)) return false;
        if (h == 0 && i >= 2 && !mbar_wait_sleep(&d_empty[db], ((i >> 1) - 1) & 1, abort_flag))
          return false;
        fence_after_sync();
        const uint32_t d = tmem + S::TM_D + (uint32_t)(db * ND);
        const uint32_t e0 = tmem + (uint32_t)(sb * S::UQ);
        const uint64_t dph = dPhiM + (uint64_t)((h * 16 * S::GRP) >> 4);
#pragma unroll
        for (int kk = 0; kk < S::UQ / 16; ++kk) {  // 16 queries (two groups) per K step
          const uint32_t eh = e0 + (uint32_t)(32 * (kk >> 1) + 8 * (kk & 1));
          const uint64_t qo = (uint64_t)((2 * kk * S::GRP) >> 4);
          mma_f16_ts(d, eh, dph + qo, IDESC2, (h > 0 || kk > 0) ? 1u : 0u);
          if constexpr (!S::MERGE) mma_f16_ts(d, eh, dph + PHI_LO + qo, IDESC2, 1u);
        }
        if (h == nh - 1) mma_commit(&d_full[db]);
        return true;
      };
      // MMA 1 runs LEAD units ahead of MMA 2 (MMAs execute in issue order, so
      // MMA 1 of unit u + LEAD overwrites buffer (u + LEAD) % NBUF only after
      // MMA 2 of unit u + LEAD - NBUF < u has read it)
      constexpr int LEAD = NBUF - 1;
      bool ok = true;
      for (int u = 0; ok && u < LEAD && u < U; ++u) ok = mma1(u);
      for (int u = 0; ok && u < U; ++u) {
        if (u + LEAD < U) ok = mma1(u + LEAD);
        if (ok) ok = mma2(u);
      }
      if (!ok) fail();
    }
  } else {
    // ---- epilogue: e = 2^S, beta' = e (dy' . w) written back in place as
    // FP16, and sum_q e dy' per candidate in FP32
    const int quad = warp & 3, grp = (warp - 4) >> 2;
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
    const int j = quad * 32 + lane;  // candidate lane
    float hsc[N];
#pragma unroll
    for (int d = 0; d < N; ++d) hsc[d] = sh[d];
    // Record part GG (positions [GG PARTW, min(RPT, (GG + 1) PARTW))) of entry
    // (candidate j, chunk ic) from D (lane j): Gc_k = -1/2 h_k dys D[k]
    // (hi + lo blocks summed), dl/dw_c = dys (sum of the two halves' e dy').
    // the chain's per-candidate stash row and sum_q e dy' (captured, so that
    // they stay in registers)
    float sv[N + 6] = {}, gw[3] = {};
    auto part = [&](int ic, auto gtag) {
      constexpr int GG = decltype(gtag)::value;
      constexpr int p0 = GG * S::PARTW;
      constexpr int p1 = (GG + 1) * S::PARTW < S::RPT ? (GG + 1) * S::PARTW : S::RPT;
      constexpr int PW = p1 - p0, PQ = PW / 4;
      constexpr unsigned long long KM0 = chain_mask_word<N>(p0, p1, 0);
      constexpr unsigned long long KM1 = chain_mask_word<N>(p0, p1, 1);
      const int db = ic & 1;
      const bool live = __float_as_int(sv[N + 3]) >= 0;
      float Gc[F];
#pragma unroll
      for (int k = 0; k < F; ++k) Gc[k] = 0.0f;
      {
        uint32_t v[KP];
#pragma unroll
        for (int b = 0; b < KP / 8; ++b) {
          bool need = false;
#pragma unroll
          for (int q = 0; q < 8; ++q) need = need || kneed(KM0, KM1, 8 * b + q);
          if (need) tmem_ld8_nowait(tmem + lane_off + S::TM_D + (uint32_t)(db * ND + 8 * b), v + 8 * b);
        }
        tmem_wait_ld();
#pragma unroll
        for (int b = 0; b < KP / 8; ++b) {
          bool need = false;
#pragma unroll
          for (int q = 0; q < 8; ++q) need = need || kneed(KM0, KM1, 8 * b + q);
          if (need) tmem_reg_fence8(v + 8 * b);
        }
#pragma unroll
        for (int k = 0; k < F; ++k)
          if (kneed(KM0, KM1, k)) Gc[k] = __uint_as_float(v[k]);
      }
      if constexpr (S::MERGE) {  // the lo block: columns KP .. 2 KP - 1
        uint32_t v[KP];
#pragma unroll
        for (int b = 0; b < KP / 8; ++b) {
          bool need = false;
#pragma unroll
          for (int q = 0; q < 8; ++q) need = need || kneed(KM0, KM1, 8 * b + q);
          if (need)
            tmem_ld8_nowait(tmem + lane_off + S::TM_D + (uint32_t)(db * ND + KP + 8 * b), v + 8 * b);
        }
        tmem_wait_ld();
#pragma unroll
        for (int b = 0; b < KP / 8; ++b) {
          bool need = false;
#pragma unroll
          for (int q = 0; q < 8; ++q) need = need || kneed(KM0, KM1, 8 * b + q);
          if (need) tmem_reg_fence8(v + 8 * b);
        }
#pragma unroll
        for (int k = 0; k < F; ++k)
          if (kneed(KM0, KM1, k)) Gc[k] += __uint_as_float(v[k]);
      }
      const float gsc = -0.5f * s_dys * sv[N + 5];
#pragma unroll
      for (int d = 0; d < N; ++d)
#pragma unroll
        for (int e = 0; e <= d; ++e)
          if (kneed(KM0, KM1, tri(d) + e)) Gc[tri(d) + e] *= gsc * (hsc[d] * hsc[e]);
#pragma unroll
      for (int d = 0; d < N; ++d)
        if (kneed(KM0, KM1, P + d)) Gc[P + d] *= gsc * hsc[d];
      Gc[P + N] *= gsc;
      const float Gc0 = Gc[P + N];
      float val[PW];
#pragma unroll
      for (int k = 0; k < PW; ++k) val[k] = 0.0f;
#pragma unroll
      for (int d = 0; d < N; ++d)
#pragma unroll
        for (int e = 0; e <= d; ++e) {
          const int p = tri(d) + e;
          if (p >= p0 && p < p1) {
            const float mi = sv[d], mk = sv[e];
            val[p - p0] = (d == e) ? Gc[p] - 2.0f * Gc[P + d] * mi + Gc0 * mi * mi
                                   : Gc[p] - (Gc[P + d] * mk + Gc[P + e] * mi) + Gc0 * mi * mk;
          }
        }
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (P + i >= p0 && P + i < p1) val[P + i - p0] = Gc0 * sv[i] - Gc[P + i];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (P + N + c >= p0 && P + N + c < p1) val[P + N + c - p0] = gw[c] * s_dys;
      if (!live) {
#pragma unroll
        for (int k = 0; k < PW; ++k) val[k] = 0.0f;
      }
      // the warp's 32 records are consecutive entries: stage 16 at a time and
      // store coalesced; entries past the tile's end are not written
      const long long w0 = beg + (long long)ic * NC + quad * 32;
      const long long nval = end - w0 < 32 ? end - w0 : 32;
      float4* stg = Outs + (warp - 4) * (16 * S::PQS);
      float4* dst = reinterpret_cast<float4*>(a.part) + w0 * S::RQT + p0 / 4;
#pragma unroll
      for (int hb = 0; hb < 2; ++hb) {
        if ((lane >> 4) == hb) {
          const int r = lane & 15;
#pragma unroll
          for (int k = 0; k < PQ; ++k)
            stg[r * S::PQS + k] =
                make_float4(val[4 * k], val[4 * k + 1], val[4 * k + 2], val[4 * k + 3]);
        }
        __syncwarp();
        const int nrec = (int)(nval - 16 * hb < 0 ? 0 : (nval - 16 * hb < 16 ? nval - 16 * hb : 16));
#pragma unroll
        for (int m = 0; m < (16 * PQ + 31) / 32; ++m) {
          const int idx = m * 32 + lane;
          const int r = idx / PQ, k = idx - r * PQ;
          if (r < nrec) dst[(long long)(16 * hb + r) * S::RQT + k] = stg[r * S::PQS + k];
        }
        __syncwarp();
      }
    };
    auto chain = [&](int ic) -> bool {
      const int db = ic & 1;
      if (!warp_wait(&gw_full[ic % SS], (ic / SS) & 1, abort_flag)) return false;
      {
        const float* sl = slot_f(ic);
#pragma unroll
        for (int k = 0; k < N + 6; ++k) sv[k] = sl[k * NC + j];
        const float4* g2 = reinterpret_cast<const float4*>(sl + NC * SV);
        const float4 ga = g2[j], gb = g2[NC + j];
        gw[0] = ga.x + gb.x;
        gw[1] = ga.y + gb.y;
        gw[2] = ga.z + gb.z;
      }
      if (!warp_wait(&d_full[db], (ic >> 1) & 1, abort_flag)) return false;
      fence_after_sync();
      // the two warps of a lane quarter form half of the parts each
      if constexpr (S::NPART > 2) {
        if (grp == 0) {
          part(ic, IntTag<0>{});
          part(ic, IntTag<1>{});
        } else {
          part(ic, IntTag<2>{});
          part(ic, IntTag<3>{});
        }
      } else {
        if (grp == 0) part(ic, IntTag<0>{});
        else part(ic, IntTag<1>{});
      }
      fence_before_sync();
      warp_arrive(&d_empty[db]);
      warp_arrive(&stash_empty[ic % SS]);
      return true;
    };
    float back = 1.0f, w0 = 0.f, w1 = 0.f, w2 = 0.f;
    float2 g0 = make_float2(0.f, 0.f), g1 = g0, g2 = g0;
    // one unit's 64 columns of this warp: e = 2^(s back), beta' to FP16 in
    // place (the first 16 columns of each 32-query block), sum_q e dy'
    auto block = [&](uint32_t col, int q0, uint32_t* v, auto sc_tag) {
      constexpr bool SC = decltype(sc_tag)::value;
      constexpr int WC = S::UQ / 2;
#pragma unroll
      for (int cb = 0; cb < WC; cb += 32) {
        uint32_t bw[16];
#pragma unroll
        for (int p = 0; p < 16; ++p) {
          const int q = q0 + cb + 2 * p;
          float2 sv2 = make_float2(__uint_as_float(v[cb + 2 * p]), __uint_as_float(v[cb + 2 * p + 1]));
          if constexpr (SC) sv2 = __fmul2_rn(sv2, make_float2(back, back));
          const float2 e = make_float2(ex2_approx(sv2.x), ex2_approx(sv2.y));
          const float2 d0 = *reinterpret_cast<const float2*>(sdyc + q);
          const float2 d1 = *reinterpret_cast<const float2*>(sdyc + 256 + q);
          const float2 d2 = *reinterpret_cast<const float2*>(sdyc + 512 + q);
          float2 tw = __fmul2_rn(d0, make_float2(w0, w0));
          tw = __ffma2_rn(d1, make_float2(w1, w1), tw);
          tw = __ffma2_rn(d2, make_float2(w2, w2), tw);
          const float2 be = __fmul2_rn(e, tw);
          g0 = __ffma2_rn(e, d0, g0);
          g1 = __ffma2_rn(e, d1, g1);
          g2 = __ffma2_rn(e, d2, g2);
          const __half2 bh = __floats2half2_rn(be.x, be.y);
          bw[p] = *reinterpret_cast<const uint32_t*>(&bh);
        }
        tmem_st16(col + (uint32_t)cb, bw);
      }
    };
    bool ok = true;
    for (int u = 0; u < U; ++u) {
      const int i = u / nh, h = u - i * nh, sb = u % NBUF;
      ok = warp_wait(&s_full[sb], (u / NBUF) & 1, abort_flag);
      if (ok && h == 0) ok = warp_wait(&stash_full[i % SS], (i / SS) & 1, abort_flag);
      if (!ok) break;
      fence_after_sync();
      if (h == 0) {
        const float* st = slot_f(i) + j;
        w0 = st[N * NC];
        w1 = st[(N + 1) * NC];
        w2 = st[(N + 2) * NC];
        back = st[(N + 4) * NC];
        g0 = g1 = g2 = make_float2(0.f, 0.f);
      }
      constexpr int WC = S::UQ / 2;
      const uint32_t col = tmem + lane_off + (uint32_t)(sb * S::UQ + grp * WC);
      const int q0 = h * S::UQ + grp * WC;  // query of column 0
      uint32_t v[WC];
#pragma unroll
      for (int cb = 0; cb < WC; cb += 16) tmem_ld16_nowait(col + (uint32_t)cb, v + cb);
      tmem_wait_ld();
#pragma unroll
      for (int cb = 0; cb < WC; cb += 16) tmem_reg_fence16(v + cb);
      // rows scaled down to fit FP16 (rare) multiply s back; a warp without
      // such a row skips the multiply
      if (__all_sync(0xffffffffu, back == 1.0f)) block(col, q0, v, BoolTag<false>{});
      else block(col, q0, v, BoolTag<true>{});
      tmem_wait_st();

      if (h == nh - 1) {
        // this warp's half of sum_q e dy' for the chunk's candidates
        float4* gd = reinterpret_cast<float4*>(slot_f(i) + NC * SV) + grp * NC + j;
        *gd = make_float4(g0.x + g0.y, g1.x + g1.y, g2.x + g2.y, 0.0f);
        warp_arrive(&gw_full[i % SS]);
      }
      fence_before_sync();
      warp_arrive(&e_full[sb]);
      // the chain of the previous chunk: its D is complete (MMA 2 of its last
      // unit ran while this chunk's units were exponentiated), and MMA 2 of
      // the next chunk waits for its buffer
      if (h == nh - 1 && i >= 1) ok = chain(i - 1);
      if (__shfl_sync(0xffffffffu, (!ok || *abort_flag) ? 1 : 0, 0)) {
        ok = false;
        break;
      }
    }
    if (ok && nchunks >= 1 && U > 0) ok = chain(nchunks - 1);
    if (!ok && lane == 0) fail();
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 12 && lane == 0) {
    // every MMA this thread issued has completed once this commit arrives
    mma_commit(&drain);
    if (!mbar_wait_bounded(&drain, 0, kWaitLimit)) fail();
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tmem, 512);
  }
}

int launch_bwd_hb(int N, const BwdArgs& a, long long T, cudaStream_t s) {
  if (T <= 0) return 0;
#define L_BB(n)                                                                         \
  {                                                                                     \
    cudaFuncSetAttribute(bwd_hb_kernel<n>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                         (int)BwdBShape<n>::SMEM);                                      \
    bwd_hb_kernel<n><<<(unsigned)T, 416, BwdBShape<n>::SMEM, s>>>(a);                   \
  }
  switch (N) {
    case 1: L_BB(1); break;
    case 2: L_BB(2); break;
    case 3: L_BB(3); break;
    case 4: L_BB(4); break;
    case 5: L_BB(5); break;
    case 6: L_BB(6); break;
    case 7: L_BB(7); break;
    case 8: L_BB(8); break;
    case 9: L_BB(9); break;
    case 10: L_BB(10); break;
    case 11: L_BB(11); break;
    case 12: L_BB(12); break;
    default: return 0;
  }
#undef L_BB
  return 1;
}

}  // namespace ndg
