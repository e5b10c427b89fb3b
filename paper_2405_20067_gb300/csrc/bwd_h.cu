// bwd_h.cu -- the analytic backward (Section 3.3) on the tensor cores with
// FP16 hi / lo operands (ndg_backward, NDG_MODE_TC, N <= 6).
//
// With the lifted form of the forward (s = phi(x~) . coef, e = 2^s, the
// coefficients scaled by -log2(e) / 2 so that de/dQ = -e / 2 for the
// quadratic form Q = (x~ - m~)^T A (x~ - m~)), every gradient of an entry
// (Gaussian j, tile) is a sum over the tile's queries q of e_jq times a
// query-side quantity:
//   dl/dc_k = -1/2 sum_c w_jc sum_q e_jq dy_qc phi_qk      (lifted coefficients)
//   dl/dw_jc = sum_q e_jq dy_qc                            (phi's constant entry)
// so after  S^T = Coef Phi^T  (MMA 1, candidates on the TMEM lanes) and
// E = 2^S, one more product  D2 = E Psi  with  Psi[q, (c, k)] = dy_qc phi_qk
// (built once per tile) yields all of them (MMA 2, A = E read straight from
// tensor memory, B = Psi from shared memory).  Per entry the kernel writes,
// in entry order (BwdArgs::slot is not used), the frame-free record
// [G = dl/dA (symmetric), v = Gc0 m~ - G_lin, dl/dw]; both remaining factors
// are linear with per-Gaussian matrices, dl/dM = 2 M sum G and dl/dm = 2 A
// sum v, and are applied once per Gaussian after the segmented sum.
//
// Precision.  MMA 1 (the exponent) takes FP16 pairs v = hi + lo for both
// operands (three products, ~22 significant bits: s needs absolute accuracy).
// MMA 2 (the gradient contraction) takes E rounded once to FP16 and Psi as a
// hi + lo pair (two products): the rounding of Psi is what the frame-free
// record amplifies (G = Gc - Gc_lin m~ - ... cancels), that of E is not; an
// FP64 emulation of the benchmark's and the tests' workloads gives per-tensor
// errors of the summed records of at most 2.4e-4 this way (1.6e-3 with Psi
// single as well, 5e-6 with all three products).  Range: features are
// scaled per tile and dimension into [-1, 1] (the coefficients take the
// inverse powers of two), dy is scaled per tile by a power of two into
// [-1, 1], and coefficient rows above 2^14 are divided by a power of two that
// the epilogue multiplies back before the exponential.
//
// CTA = one tile of up to 256 queries = up to two units of 128 queries,
// 416 threads, one CTA per SM (all 512 TMEM columns):
//   warps 0-3   builders: coefficient rows of a chunk of 128 candidates into
//               one of CS stages (as in the forward), one arrival per warp;
//               after building chunk i they run the chain of chunk i - 2
//               (thread j = candidate j = TMEM lane j of the D2 buffer), so
//               that the epilogue only forms E;
//   warp 12     MMA issuer (lane 0): MMA 1 of unit u + 1, then MMA 2 of unit u
//               (TMEM: S / E buffers u & 1 at columns 128 (u & 1); D2 buffers
//               i & 1 at 256 + NPSI (i & 1), accumulated over the chunk's units);
//   warps 4-11  epilogue: warp w owns lanes 32 (w % 4) .. + 31 and columns
//               64 ((w - 4) / 4) .. + 63 of each unit: e = 2^s written back in
//               place as FP16 (32 S columns -> 16 columns of packed pairs, at
//               the first 16 of the 32).
// Every wait is bounded; a timeout records NDG_ERR_TIMEOUT and the CTA lets
// its issued MMAs finish (bounded) before it frees tensor memory.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "kernels.h"
#include "tcgen05.cuh"

namespace ndg {

template <int N>
struct BwdHShape {
  static constexpr int P = tri(N);
  static constexpr int F = P + N + 1;
  static constexpr int KP = (F + 15) / 16 * 16;
  static constexpr int NC = 128;            // candidates per chunk (MMA 1 M, TMEM lanes)
  static constexpr int NPSI = 3 * KP;       // MMA 2 N: (colour, feature)
  static constexpr int R = rec_floats(N);   // record head: A, m, w
  static constexpr int R2 = rec_tc_floats(N);
  static constexpr int RP = part_floats(N);
  static constexpr int RPT = RP;                       // per-entry record floats
  static constexpr int RQT = RPT / 4;
  static constexpr int SPLIT = (RPT / 2 + 3) / 4 * 4;  // record floats [0, SPLIT) by group 0
  static constexpr int PQMAX = (SPLIT > RPT - SPLIT ? SPLIT : RPT - SPLIT) / 4;
  static constexpr int CS = 3;              // coefficient stages
  static constexpr uint32_t SBO_K = (KP / 8) * 128;   // rows of KP FP16 values
  static constexpr uint32_t SBO_Q = (256 / 8) * 128;  // Psi rows of 256 queries
  static constexpr uint32_t PHI_BYTES = 256u * KP * 2;
  // queries per unit (MMA 1 N, MMA 2 K).  128: two S / E buffers, MMA 1 one
  // unit ahead of MMA 2.  (64 with four buffers, MMA 1 three units ahead,
  // measured 27% slower: an MMA's cost has a floor of ~46 cycles, so the
  // narrower MMA 1 and the doubled per-unit overheads outweigh the slack.)
  static constexpr int UQ = 128;
  static constexpr int NBUF = 256 / UQ;     // S / E buffers in TMEM columns [0, 256)
  static constexpr uint32_t UNIT_BYTES = (uint32_t)UQ * KP * 2;  // Phi rows of one unit
  static constexpr uint32_t PSI_BYTES = (uint32_t)NPSI * 256 * 2;
  static constexpr uint32_t C_BYTES = (uint32_t)NC * KP * 2;
  static constexpr uint32_t STASH = 48;  // per candidate: m~ (N), w (3), live flag, pad
  static constexpr uint32_t C_STAGE = 2 * C_BYTES + NC * 4 + NC * STASH;  // hi, lo, row factors, stash
  // per builder warp: one half of 16 records staged for coalesced stores
  // (stride PQMAX + 1 float4 against bank conflicts)
  static constexpr uint32_t OUT_BYTES = 16u * (PQMAX + 1) * 16;
  static constexpr uint32_t SMEM_USED =
      2 * PHI_BYTES + 2 * PSI_BYTES + CS * C_STAGE + 4 * OUT_BYTES + 128;
  static constexpr uint32_t SMEM = SMEM_USED > 116u * 1024u ? SMEM_USED : 116u * 1024u;
  static constexpr uint32_t TM_D2 = 256;
  static_assert(256 + 2 * NPSI <= 512, "tensor memory");
  static_assert(SMEM <= 227u * 1024u, "shared memory");
  static_assert(NPSI % 16 == 0 && NPSI <= 256, "MMA 2 shape");
  static_assert(RPT >= P + N + 3 && N + 4 <= 12, "record / stash");
};

// Which lifted-coefficient gradients Gc_k (bit k) a group of the chain needs
// for its record positions [p0, p1): G (i, k) needs Gc_ik, Gc_lin_i, Gc_lin_k
// and Gc0; v_i needs Gc_lin_i and Gc0; dl/dw needs the constant column.
template <int N>
__host__ __device__ constexpr uint32_t chain_kmask(int p0, int p1) {
  constexpr int P = tri(N);
  uint32_t m = 0;
  for (int d = 0; d < N; ++d)
    for (int e = 0; e <= d; ++e) {
      const int p = tri(d) + e;
      if (p >= p0 && p < p1) m |= (1u << p) | (1u << (P + d)) | (1u << (P + e)) | (1u << (P + N));
    }
  for (int i = 0; i < N; ++i)
    if (P + i >= p0 && P + i < p1) m |= (1u << (P + i)) | (1u << (P + N));
  for (int c = 0; c < 3; ++c)
    if (P + N + c >= p0 && P + N + c < p1) m |= 1u << (P + N);
  return m;
}

namespace {

__device__ __forceinline__ void split_h2b(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(v0, v1);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(v0 - hf.x, v1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ uint32_t koff(int row, int k, uint32_t sbo) {
  return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k & 7) * 2u;
}

template <int KP>
__device__ __forceinline__ void store_row_hb(uint8_t* hi, uint8_t* lo, int row, uint32_t sbo,
                                             const float (&v)[KP]) {
#pragma unroll
  for (int k = 0; k < KP; k += 8) {
    uint4 h, l;
    split_h2b(v[k], v[k + 1], h.x, l.x);
    split_h2b(v[k + 2], v[k + 3], h.y, l.y);
    split_h2b(v[k + 4], v[k + 5], h.z, l.z);
    split_h2b(v[k + 6], v[k + 7], h.w, l.w);
    const uint32_t off = koff(row, k, sbo);
    *reinterpret_cast<uint4*>(hi + off) = h;
    *reinterpret_cast<uint4*>(lo + off) = l;
  }
}

constexpr float kNegHalfLog2eB = -0.72134752044448170368f;
constexpr float kRowMaxB = 16384.0f;

}  // namespace

template <int N>
__global__ void __launch_bounds__(416, 1) bwd_h_kernel(BwdArgs a) {
  using S = BwdHShape<N>;
  constexpr int P = S::P, F = S::F, KP = S::KP, NC = S::NC, NPSI = S::NPSI, CS = S::CS;
  constexpr int R4 = S::R / 4, R2 = S::R2;
  extern __shared__ __align__(128) uint8_t dsm[];
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm + 127) & ~(uintptr_t)127);
  uint8_t* PhiH = base;
  uint8_t* PhiL = PhiH + S::PHI_BYTES;
  uint8_t* PsiH = PhiL + S::PHI_BYTES;
  uint8_t* PsiL = PsiH + S::PSI_BYTES;
  uint8_t* Cst = PsiL + S::PSI_BYTES;  // CS stages of (hi, lo, row factors)
  float4* Outs = reinterpret_cast<float4*>(Cst + CS * S::C_STAGE);  // 4 x OUT_BYTES
  __shared__ uint64_t coef_full[CS], coef_empty[CS], s_full[S::NBUF], e_full[S::NBUF], d2_full[2], d2_empty[2],
      drain;
  __shared__ uint32_t tmem_base;
  __shared__ float sred[8 * N * 2], sdy[8];
  __shared__ float sctr[N], sh[N], s_dys;
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long t = blockIdx.x;
  const long long qt = t * a.tile;
  const int nq = (int)(a.Q - qt < a.tile ? a.Q - qt : a.tile);
  const int nh = (nq + S::UQ - 1) / S::UQ;  // units (blocks of UQ queries) per chunk

  if (tid == 0) {
    for (int i = 0; i < CS; ++i) {
      mbar_init(&coef_full[i], 4);
      mbar_init(&coef_empty[i], 1 + 8 + 4);  // MMA 1, epilogue warps, builders' chain
    }
    for (int i = 0; i < S::NBUF; ++i) {
      mbar_init(&s_full[i], 1);
      mbar_init(&e_full[i], 8);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&d2_full[i], 1);
      mbar_init(&d2_empty[i], 4);
    }
    mbar_init(&drain, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  // ---- per tile: centre, feature and dy scales, Phi rows and Psi columns
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
    store_row_hb<KP>(PhiH, PhiL, row, S::SBO_K, phi);
    const float idys = 1.0f / s_dys;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float dc = dq[c] * idys;
#pragma unroll
      for (int k = 0; k < KP; k += 2) {
        uint32_t hv, lv;
        split_h2b(dc * phi[k], dc * phi[k + 1], hv, lv);
        const int r = c * KP + k;  // rows r and r + 1, K index = query `row`
        *reinterpret_cast<uint16_t*>(PsiH + koff(r, row, S::SBO_Q)) = (uint16_t)(hv & 0xffffu);
        *reinterpret_cast<uint16_t*>(PsiH + koff(r + 1, row, S::SBO_Q)) = (uint16_t)(hv >> 16);
        *reinterpret_cast<uint16_t*>(PsiL + koff(r, row, S::SBO_Q)) = (uint16_t)(lv & 0xffffu);
        *reinterpret_cast<uint16_t*>(PsiL + koff(r + 1, row, S::SBO_Q)) = (uint16_t)(lv >> 16);
      }
    }
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

  if (warp < 4) {
    // ---- builders (thread j = candidate j of each chunk); the records of
    // chunk i + 1 are loaded into registers while chunk i is built
    const int j = tid;
    float hsc[N];
#pragma unroll
    for (int d = 0; d < N; ++d) hsc[d] = sh[d];
    // candidate j of chunk i: Gaussian index (or -1) and its entry index (or -1)
    auto cand = [&](int i) -> int2 {
      const long long e = beg + (long long)i * NC + j;
      const bool in = i < nchunks && e < end;
      const int g = in ? a.ids[e] : -1;
      const bool live = (unsigned)g < (unsigned)a.Ge;
      const int sl = live ? (int)e : -1;
      return make_int2(live ? g : -1, sl);
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
      float buf[S::R];
#pragma unroll
      for (int k = 0; k < R4; ++k) {
        buf[4 * k] = cur[k].x; buf[4 * k + 1] = cur[k].y;
        buf[4 * k + 2] = cur[k].z; buf[4 * k + 3] = cur[k].w;
      }
      if (i >= CS && !warp_wait(&coef_empty[s], ((i / CS) - 1) & 1, abort_flag)) return false;
      uint8_t* st = Cst + s * S::C_STAGE;
      float coef[KP], mt[N];
#pragma unroll
      for (int d = 0; d < N; ++d) mt[d] = buf[P + d] - sctr[d];
      float cst = 0.0f;
#pragma unroll
      for (int d = 0; d < N; ++d) {
        float s2 = 0.0f;
#pragma unroll
        for (int k = 0; k < N; ++k) s2 = fmaf(buf[d >= k ? tri(d) + k : tri(k) + d], mt[k], s2);
        coef[P + d] = (kNegHalfLog2eB * -2.0f) * s2 * hsc[d];
        cst = fmaf(mt[d], s2, cst);
      }
#pragma unroll
      for (int d = 0; d < N; ++d)
#pragma unroll
        for (int k = 0; k <= d; ++k)
          coef[tri(d) + k] = kNegHalfLog2eB * (d == k ? buf[tri(d) + k] : 2.0f * buf[tri(d) + k]) *
                             (hsc[d] * hsc[k]);
      coef[P + N] = kNegHalfLog2eB * cst;
#pragma unroll
      for (int k = F; k < KP; ++k) coef[k] = 0.0f;
      float mx = 0.0f;
#pragma unroll
      for (int k = 0; k < F; ++k) mx = fmaxf(mx, fabsf(coef[k]));
      float back = 1.0f;
      if (mx > kRowMaxB) {
        int ex = (int)((__float_as_uint(mx) >> 23) & 0xffu) - 127 - 13;
        ex = ex > 120 ? 120 : ex;
        const float down = __uint_as_float((uint32_t)(127 - ex) << 23);
        back = __uint_as_float((uint32_t)(127 + ex) << 23);
#pragma unroll
        for (int k = 0; k < KP; ++k) coef[k] *= down;
      }
      store_row_hb<KP>(st, st + S::C_BYTES, j, S::SBO_K, coef);
      reinterpret_cast<float*>(st + 2 * S::C_BYTES)[j] = back;
      {
        // what the chain of this entry needs: m~, w and whether it is live
        float sv[12];
#pragma unroll
        for (int d = 0; d < N; ++d) sv[d] = mt[d];
#pragma unroll
        for (int c = 0; c < 3; ++c) sv[N + c] = buf[P + N + c];
        sv[N + 3] = __int_as_float(slot);
#pragma unroll
        for (int k = N + 4; k < 12; ++k) sv[k] = 0.0f;
        float4* dst = reinterpret_cast<float4*>(st + 2 * S::C_BYTES + NC * 4 + (uint32_t)j * S::STASH);
        dst[0] = make_float4(sv[0], sv[1], sv[2], sv[3]);
        dst[1] = make_float4(sv[4], sv[5], sv[6], sv[7]);
        dst[2] = make_float4(sv[8], sv[9], sv[10], sv[11]);
      }
      fence_proxy_async();
      warp_arrive(&coef_full[s]);
      return true;
    };
    // Chain of entry (candidate j, chunk ic).  From D2 = sum_q e dy' phi' the
    // gradient with respect to the unscaled lifted coefficients is
    // Gc_k = -1/2 h_k dys sum_c w_c D2[c][k] and dl/dw_c = dys D2[c][P + N]
    // (the constant feature); the record is the frame-free [G = dl/dA
    // (symmetric, lower packed), v = Gc0 m~ - G_lin, dl/dw] (dl/dM = 2 M sum G
    // and dl/dm = 2 A sum v follow per Gaussian).  The record is formed in two
    // halves of positions (fewer live registers), each loading only the D2
    // columns it needs.
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    auto half = [&](int ic, const float (&sv)[12], auto gtag) {
      constexpr int GG = decltype(gtag)::value;
      constexpr int RPT = S::RPT, SPLIT = S::SPLIT;
      constexpr int p0 = GG ? SPLIT : 0, p1 = GG ? RPT : SPLIT, PW = p1 - p0, PQ = PW / 4;
      const int db = ic & 1;
      const bool live = __float_as_int(sv[N + 3]) >= 0;
      constexpr uint32_t KM = chain_kmask<N>(p0, p1);  // needed Gc_k (F <= 28 bits)
      float Gc[F], gw[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < F; ++k) Gc[k] = 0.0f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        uint32_t v[KP];
#pragma unroll
        for (int b = 0; b < KP / 8; ++b)
          if ((KM >> (8 * b)) & 0xffu)
            tmem_ld8_nowait(tmem + lane_off + S::TM_D2 + (uint32_t)(db * NPSI + c * KP + 8 * b), v + 8 * b);
        tmem_wait_ld();
#pragma unroll
        for (int b = 0; b < KP / 8; ++b)
          if ((KM >> (8 * b)) & 0xffu) tmem_reg_fence8(v + 8 * b);
        const float wc = sv[N + c];
#pragma unroll
        for (int k = 0; k < F; ++k)
          if ((KM >> k) & 1u) Gc[k] = fmaf(wc, __uint_as_float(v[k]), Gc[k]);
        gw[c] = __uint_as_float(v[P + N]);
      }
      const float gsc = -0.5f * s_dys;
#pragma unroll
      for (int d = 0; d < N; ++d)
#pragma unroll
        for (int e = 0; e <= d; ++e)
          if ((KM >> (tri(d) + e)) & 1u) Gc[tri(d) + e] *= gsc * (hsc[d] * hsc[e]);
#pragma unroll
      for (int d = 0; d < N; ++d)
        if ((KM >> (P + d)) & 1u) Gc[P + d] *= gsc * hsc[d];
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
      // The warp's 32 records are consecutive entries: stage this half of 16
      // records at a time and store with coalesced accesses; entries past the
      // tile's end are not written.
      const long long w0 = beg + (long long)ic * NC + warp * 32;
      const long long nval = end - w0 < 32 ? end - w0 : 32;
      float4* stg = Outs + warp * (16 * (S::PQMAX + 1));
      float4* dst = reinterpret_cast<float4*>(a.part) + w0 * S::RQT + p0 / 4;
#pragma unroll
      for (int hb = 0; hb < 2; ++hb) {
        if ((lane >> 4) == hb) {
          const int r = lane & 15;
#pragma unroll
          for (int k = 0; k < PQ; ++k)
            stg[r * (S::PQMAX + 1) + k] =
                make_float4(val[4 * k], val[4 * k + 1], val[4 * k + 2], val[4 * k + 3]);
        }
        __syncwarp();
        const int nrec = (int)(nval - 16 * hb < 0 ? 0 : (nval - 16 * hb < 16 ? nval - 16 * hb : 16));
#pragma unroll
        for (int m = 0; m < (16 * PQ + 31) / 32; ++m) {
          const int idx = m * 32 + lane;
          const int r = idx / PQ, k = idx - r * PQ;
          if (r < nrec) dst[(long long)(16 * hb + r) * S::RQT + k] = stg[r * (S::PQMAX + 1) + k];
        }
        __syncwarp();
      }
    };
    auto chain = [&](int ic) -> bool {
      const int db = ic & 1, s = ic % CS;
      float sv[12];
      {
        const float4* stp = reinterpret_cast<const float4*>(Cst + s * S::C_STAGE + 2 * S::C_BYTES +
                                                            NC * 4 + (uint32_t)j * S::STASH);
        const float4 v0 = stp[0], v1 = stp[1], v2 = stp[2];
        sv[0] = v0.x; sv[1] = v0.y; sv[2] = v0.z; sv[3] = v0.w;
        sv[4] = v1.x; sv[5] = v1.y; sv[6] = v1.z; sv[7] = v1.w;
        sv[8] = v2.x; sv[9] = v2.y; sv[10] = v2.z; sv[11] = v2.w;
      }
      warp_arrive(&coef_empty[s]);
      if (!warp_wait(&d2_full[db], (ic >> 1) & 1, abort_flag)) return false;
      fence_after_sync();
      half(ic, sv, IntTag<0>{});
      half(ic, sv, IntTag<1>{});
      fence_before_sync();
      warp_arrive(&d2_empty[db]);
      return true;
    };
    float4 cur[R4], nxt[R4];
    const int2 c0i = cand(0);
    load(c0i.x, cur);
    int slot_cur = c0i.y;
    int2 c_next = cand(1);
    bool ok = true;
    for (int i = 0; i < nchunks; ++i) {
      load(c_next.x, nxt);
      const int slot_nxt = c_next.y;
      c_next = cand(i + 2);
      ok = build(i, cur, slot_cur);
      slot_cur = slot_nxt;
#pragma unroll
      for (int k = 0; k < R4; ++k) cur[k] = nxt[k];
      // the chain of chunk i - 2 (its D2 buffer is the one chunk i will use)
      if (ok && i >= 2) ok = chain(i - 2);
      if (__shfl_sync(0xffffffffu, (!ok || *abort_flag) ? 1 : 0, 0)) {
        ok = false;
        break;
      }
    }
    for (int ic = nchunks >= 2 ? nchunks - 2 : 0; ok && ic < nchunks; ++ic) ok = chain(ic);
    if (!ok && lane == 0) fail();
  } else if (warp == 12) {
    // ---- MMA issuer
    if (lane == 0 && U > 0) {
      constexpr uint32_t IDESC1 = idesc_f16(S::UQ);
      constexpr uint32_t IDESC2 = idesc_f16(NPSI);
      // descriptor bases (a descriptor for base + off is base + off / 16)
      const uint64_t dPhi = smem_desc(smem_u32(PhiH), 128, S::SBO_K);
      const uint64_t dPsi = smem_desc(smem_u32(PsiH), 128, S::SBO_Q);
      const uint64_t dC0 = smem_desc(smem_u32(Cst), 128, S::SBO_K);
      constexpr uint64_t PHI_LO = S::PHI_BYTES >> 4, PSI_LO = S::PSI_BYTES >> 4;
      constexpr uint64_t C_LO = S::C_BYTES >> 4;
      auto mma1 = [&](int u) -> bool {
        const int i = u / nh, h = u - i * nh, s = i % CS, sb = u % S::NBUF;
        if (h == 0 && !mbar_wait_sleep(&coef_full[s], (i / CS) & 1, abort_flag)) return false;
        fence_after_sync();
        const uint64_t dch = dC0 + (uint64_t)((s * S::C_STAGE) >> 4);
        const uint64_t dph = dPhi + (uint64_t)((h * S::UNIT_BYTES) >> 4);
        const uint32_t d = tmem + (uint32_t)(sb * S::UQ);
#pragma unroll
        for (int ks = 0; ks < KP / 16; ++ks) {
          const uint64_t ko = (uint64_t)ks * 16u;  // 256 bytes per K step
          mma_f16(d, dch + ko, dph + ko, IDESC1, ks > 0 ? 1u : 0u);
          mma_f16(d, dch + ko, dph + PHI_LO + ko, IDESC1, 1u);
          mma_f16(d, dch + C_LO + ko, dph + ko, IDESC1, 1u);
        }
        mma_commit(&s_full[sb]);
        if (h == nh - 1) mma_commit(&coef_empty[s]);
        return true;
      };
      auto mma2 = [&](int u) -> bool {
        const int i = u / nh, h = u - i * nh, sb = u % S::NBUF, db = i & 1;
        if (!mbar_wait_sleep(&e_full[sb], (u / S::NBUF) & 1, abort_flag)) return false;
        if (h == 0 && i >= 2 && !mbar_wait_sleep(&d2_empty[db], ((i >> 1) - 1) & 1, abort_flag))
          return false;
        fence_after_sync();
        const uint32_t d = tmem + S::TM_D2 + (uint32_t)(db * NPSI);
        const uint32_t e0 = tmem + (uint32_t)(sb * S::UQ);
        const uint64_t dsh = dPsi + (uint64_t)((S::UQ / 8) * h) * 8u;  // 128 B per 8 queries
#pragma unroll
        for (int kk = 0; kk < S::UQ / 16; ++kk) {  // 16 queries per K step
          const uint32_t eh = e0 + (uint32_t)(32 * (kk >> 1) + 8 * (kk & 1));
          const uint64_t qo = (uint64_t)(2 * kk) * 8u;
          mma_f16_ts(d, eh, dsh + qo, IDESC2, (h > 0 || kk > 0) ? 1u : 0u);
          mma_f16_ts(d, eh, dsh + PSI_LO + qo, IDESC2, 1u);
        }
        if (h == nh - 1) mma_commit(&d2_full[db]);
        return true;
      };
      // MMA 1 runs NBUF - 1 units ahead of MMA 2 (MMAs execute in issue
      // order, so MMA 1 of unit u + NBUF - 1 overwrites buffer (u - 1) % NBUF
      // only after MMA 2 of unit u - 1 has read it)
      constexpr int LEAD = S::NBUF - 1;
      bool ok = true;
      for (int u = 0; ok && u < LEAD && u < U; ++u) ok = mma1(u);
      for (int u = 0; ok && u < U; ++u) {
        if (u + LEAD < U) ok = mma1(u + LEAD);
        if (ok) ok = mma2(u);
      }
      if (!ok) fail();
    }
  } else {
    // ---- epilogue: E = 2^S written back in place as FP16
    const int quad = warp & 3, grp = (warp - 4) >> 2;
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
    const int j = quad * 32 + lane;  // candidate lane
    float hsc[N];
#pragma unroll
    for (int d = 0; d < N; ++d) hsc[d] = sh[d];
    float back = 1.0f;
    // one unit's UQ / 2 columns of this warp: E = 2^(s back) to FP16 in place
    auto block = [&](uint32_t col, uint32_t* v, auto sc_tag) {
      constexpr bool SC = decltype(sc_tag)::value;
      constexpr int WC = S::UQ / 2;
#pragma unroll
      for (int cb = 0; cb < WC; cb += 32) {
        uint32_t hi[16];
#pragma unroll
        for (int p = 0; p < 16; ++p) {
          float2 sv = make_float2(__uint_as_float(v[cb + 2 * p]), __uint_as_float(v[cb + 2 * p + 1]));
          if constexpr (SC) sv = __fmul2_rn(sv, make_float2(back, back));
          const __half2 e2 = __floats2half2_rn(ex2_approx(sv.x), ex2_approx(sv.y));
          hi[p] = *reinterpret_cast<const uint32_t*>(&e2);
        }
        tmem_st16(col + (uint32_t)cb, hi);
      }
    };
    bool ok = true;
    for (int u = 0; u < U; ++u) {
      const int i = u / nh, h = u - i * nh, s = i % CS, sb = u % S::NBUF;
      ok = warp_wait(&s_full[sb], (u / S::NBUF) & 1, abort_flag);
      if (ok && h == 0) ok = warp_wait(&coef_full[s], (i / CS) & 1, abort_flag);
      if (!ok) break;
      fence_after_sync();
      if (h == 0) {
        back = reinterpret_cast<const float*>(Cst + s * S::C_STAGE + 2 * S::C_BYTES)[j];
        warp_arrive(&coef_empty[s]);
      }
      // all UQ / 2 columns of this warp in flight at once, one wait
      constexpr int WC = S::UQ / 2;
      const uint32_t col = tmem + lane_off + (uint32_t)(sb * S::UQ + grp * WC);
      uint32_t v[WC];
#pragma unroll
      for (int cb = 0; cb < WC; cb += 16) tmem_ld16_nowait(col + (uint32_t)cb, v + cb);
      tmem_wait_ld();
#pragma unroll
      for (int cb = 0; cb < WC; cb += 16) tmem_reg_fence16(v + cb);
      // rows scaled down to fit FP16 (rare) multiply s back; a warp without
      // such a row skips the multiply
      if (__all_sync(0xffffffffu, back == 1.0f)) block(col, v, BoolTag<false>{});
      else block(col, v, BoolTag<true>{});
      tmem_wait_st();
      fence_before_sync();
      warp_arrive(&e_full[sb]);
      if (__shfl_sync(0xffffffffu, *abort_flag ? 1 : 0, 0)) {
        ok = false;
        break;
      }
    }
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

int launch_bwd_h(int N, const BwdArgs& a, long long T, cudaStream_t s) {
  if (T <= 0) return 0;
#define L_BH(n)                                                                         \
  {                                                                                     \
    cudaFuncSetAttribute(bwd_h_kernel<n>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                         (int)BwdHShape<n>::SMEM);                                      \
    bwd_h_kernel<n><<<(unsigned)T, 416, BwdHShape<n>::SMEM, s>>>(a);                    \
  }
  switch (N) {
    case 1: L_BH(1); break;
    case 2: L_BH(2); break;
    case 3: L_BH(3); break;
    case 4: L_BH(4); break;
    case 5: L_BH(5); break;
    case 6: L_BH(6); break;
    default: return 0;
  }
#undef L_BH
  return 1;
}

}  // namespace ndg
