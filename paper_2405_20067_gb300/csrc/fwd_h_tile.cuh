// fwd_h_tile.cuh -- lifted-feature evaluation on the tensor cores with FP16
// operands split into high and low halves (ndg_forward, NDG_MODE_TC).
//
// Same quadratic-form evaluation as the TF32 kernels: for a tile with centre
// c the exponent of Eq. 1 is  s = phi(x~) . coef  with lifted features
// phi = [x~_i x~_j (j <= i), x~_i, 1] and per-(Gaussian, tile) coefficients
// coef = [A_ii | 2 A_ij, -2 A m~, m~^T A m~] * (-log2(e) / 2), A = M^T M.
// Here the operands are FP16 pairs v = hi + lo (11 + 11 significant bits,
// three products hi hi + hi lo + lo hi accumulated in FP32), which runs at
// twice the TF32 rate and halves the operand bytes.  FP16 has a narrow
// exponent range, so both sides are rescaled by powers of two (exact):
//   * per tile and dimension, x~_d is divided by h_d = 2^ceil(log2 half-extent),
//     so the features lie in [-1, 1];  the coefficients take the inverse
//     factors (h_i h_j for the quadratic terms, h_i for the linear ones);
//   * per candidate, a row whose largest coefficient exceeds 2^14 is divided
//     by 2^k; the epilogue multiplies the accumulator back by 2^k (the
//     stage carries a flag so that chunks without such rows skip it).
//
// CTA = one tile of up to 256 queries (two M = 128 row blocks sharing the
// candidate operand), 416 threads, one CTA per SM (it owns all 512 TMEM
// columns: two accumulator buffers x two row blocks x 128 candidates):
//   warps 0-3   builders: thread j turns candidate j of a chunk of 128 into
//               its coefficient row (FP16 hi / lo, K-major no-swizzle layout)
//               and weight pair entry in one of CS shared-memory stages; the
//               records of the next chunk are loaded into registers meanwhile;
//               each warp then arrives on coef_full;
//   warp 12     MMA issuer: lane 0 issues the MMAs of chunk i once its stage
//               is full and accumulator buffer i & 1 is free, and commits
//               them to acc_full and coef_empty (a warp of its own, so that
//               issuing overlaps the building of the next chunks);
//   warps 4-11  epilogue: warps 4-7 serve row block 0, warps 8-11 row block 1
//               (each block has its own accumulator barriers, so the two
//               groups run independently); warp w reads TMEM lanes 32 (w % 4)
//               .. + 31 of its block at all 128 columns with the 16x256b load
//               shape (a thread holds 4 rows x 2 columns of every 8-column
//               group), the loads of the next 32 columns in flight while the
//               current ones are used; it forms e = 2^s and accumulates w e;
//               row sums are completed with shuffles at the end.
// Barrier operations are one per warp (an elected lane), and every wait is
// bounded: on a timeout the kernel records NDG_ERR_TIMEOUT, lets the issued
// MMAs finish (bounded), frees its tensor memory and returns.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "kernels.h"
#include "tcgen05.cuh"

namespace ndg {

template <int N>
struct FwdHShape {
  static constexpr int P = tri(N);
  static constexpr int F = P + N + 1;
  static constexpr int KP = (F + 15) / 16 * 16;  // K step of kind::f16 is 16
  static constexpr int NC = 128;                 // candidates per chunk (MMA N)
  static constexpr int R = rec_floats(N);
  static constexpr uint32_t SBO = (KP / 8) * 128;  // 8-row group stride (bytes)
  static constexpr uint32_t PHI_BYTES = 256u * KP * 2;  // one of hi / lo, 256 rows
  static constexpr uint32_t HALF_BYTES = 128u * KP * 2; // one 128-row block
  static constexpr uint32_t B_BYTES = (uint32_t)NC * KP * 2;
  static constexpr uint32_t W_BYTES = (uint32_t)NC * 16;  // w0 w0' w1 w1' w2 w2' k k' per pair
  static constexpr uint32_t C_STAGE = 2 * B_BYTES + W_BYTES;
  // coefficient stages: as many as fit next to Phi (at most 4; 2 KB are left
  // for the static shared variables).  The builders run up to CS chunks ahead
  // of the epilogue, which frees a stage only at the end of its chunk, so
  // two stages leave the builders idle for a whole chunk (measured at N = 10:
  // a third stage is worth about a fifth of the time).
  static constexpr uint32_t STAGE_ROOM = 227u * 1024u - 2048u - 2 * PHI_BYTES - 128u;
  static constexpr int CS = STAGE_ROOM / C_STAGE >= 4 ? 4 : (int)(STAGE_ROOM / C_STAGE);
  static constexpr uint32_t SMEM_USED = 2 * PHI_BYTES + CS * C_STAGE + 128;
  // more than half of the SM's shared memory: one CTA per SM
  static constexpr uint32_t SMEM = SMEM_USED > 116u * 1024u ? SMEM_USED : 116u * 1024u;
  static_assert(SMEM <= 227u * 1024u, "shared memory");
  static_assert(CS >= 2, "coefficient stages");
  static_assert(NC == 128, "candidate mapping");
};

namespace {

// Splits (v0, v1) into FP16 high and low halves, packed as half2 words.
__device__ __forceinline__ void split_h2(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(v0, v1);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(v0 - hf.x, v1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Byte offset of element (row, k) of a K-major no-swizzle FP16 operand.
__device__ __forceinline__ uint32_t kmajor_off_h(int row, int k, uint32_t sbo) {
  return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k & 7) * 2u;
}

// Writes one K-major row of KP values (multiple of 8) as FP16 hi / lo.
template <int KP>
__device__ __forceinline__ void store_row_h(uint8_t* hi, uint8_t* lo, int row, uint32_t sbo,
                                            const float (&v)[KP]) {
#pragma unroll
  for (int k = 0; k < KP; k += 8) {
    uint4 h, l;
    split_h2(v[k], v[k + 1], h.x, l.x);
    split_h2(v[k + 2], v[k + 3], h.y, l.y);
    split_h2(v[k + 4], v[k + 5], h.z, l.z);
    split_h2(v[k + 6], v[k + 7], h.w, l.w);
    const uint32_t off = kmajor_off_h(row, k, sbo);
    *reinterpret_cast<uint4*>(hi + off) = h;
    *reinterpret_cast<uint4*>(lo + off) = l;
  }
}

constexpr float kNegHalfLog2eH = -0.72134752044448170368f;
constexpr float kRowMax = 16384.0f;  // coefficient rows are kept below 2^14 (FP16 max 65504)

}  // namespace

// Barriers and small shared state of one tile, sized for the largest shape
// (CS <= 4 coefficient stages, N <= 12).
struct FwdHSync {
  // accumulator barriers per (buffer, row block): index 2 b + h
  uint64_t coef_full[4], coef_empty[4], acc_full[4], acc_empty[4], drain;
  uint32_t tmem_base;
  float sred[8 * 12 * 2];
  float sctr[12], sh[12];
  __align__(16) int sflag[4][4];
  int s_abort;
};

// Query tile t on the tensor cores, by the whole CTA.  The caller owns the
// tensor memory (all 512 columns, address in sy.tmem_base, visible after
// the tile's first block barrier).  Returns after a block barrier with every
// MMA of the tile complete, so that the caller may start another tile.
template <int N>
__device__ __forceinline__ void fwd_tile(const FwdArgs& a, long long t, uint8_t* base,
                                         FwdHSync& sy) {
  using S = FwdHShape<N>;
  constexpr int P = S::P, KP = S::KP, NC = S::NC, CS = S::CS, R = S::R, R4 = R / 4;
  static_assert(CS <= 4 && N <= 12, "FwdHSync sizes");
  uint8_t* Ahi = base;
  uint8_t* Alo = Ahi + S::PHI_BYTES;
  uint8_t* Cst = Alo + S::PHI_BYTES;  // CS stages of (Bhi, Blo, weights)
  uint64_t* coef_full = sy.coef_full;
  uint64_t* coef_empty = sy.coef_empty;
  uint64_t* acc_full = sy.acc_full;
  uint64_t* acc_empty = sy.acc_empty;
  uint64_t& drain = sy.drain;
  float* sred = sy.sred;
  float* sctr = sy.sctr;
  float* sh = sy.sh;
  auto& sflag = sy.sflag;
  int& s_abort = sy.s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long qt = t * a.tile;
  const int nq = (int)(a.Q - qt < a.tile ? a.Q - qt : a.tile);
  const int nh = nq > 128 ? 2 : 1;  // row blocks with queries

  // ---- setup: barriers, tile centre and scales, Phi rows (epilogue warps)
  if (tid == 0) {
    for (int i = 0; i < CS; ++i) {
      mbar_init(&coef_full[i], 4);
      mbar_init(&coef_empty[i], 1 + 4 * nh);  // issuer commit + the busy epilogue warps
    }
    for (int i = 0; i < 4; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 4);
    }
    mbar_init(&drain, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const int row = tid - 128;  // epilogue threads: Phi row
  const bool is_epi = warp >= 4 && warp < 12;
  const bool active_row = is_epi && row < nq;
  float xq[N];
#pragma unroll
  for (int d = 0; d < N; ++d) xq[d] = active_row ? a.x[(qt + row) * N + d] : 0.0f;
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
    for (int k = P + N + 1; k < KP; ++k) phi[k] = 0.0f;
    store_row_h<KP>(Ahi, Alo, row, S::SBO, phi);
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = sy.tmem_base;
  const long long beg = a.offsets[t], end = a.offsets[t + 1];
  const int nchunks = (int)((end - beg + NC - 1) / NC);
  volatile int* abort_flag = &s_abort;
  auto fail = [&]() {
    atomicExch(&s_abort, 1);
    if (a.status) set_status(a.status, NDG_ERR_TIMEOUT);
  };

  if (warp < 4) {
    // ---- builders
    const int j = tid;
    float hsc[N];
#pragma unroll
    for (int d = 0; d < N; ++d) hsc[d] = sh[d];
    auto cand = [&](int i) -> int {
      const long long c = beg + (long long)i * NC + j;
      const int g = (i < nchunks && c < end) ? a.ids[c] : -1;
      return ((unsigned)g < (unsigned)a.Ge) ? g : -1;
    };
    const int stride4 = a.rec_stride4 > 0 ? a.rec_stride4 : R4;
    auto load = [&](int g, float4 (&r)[R4]) {
      if (g >= 0) {
        const float4* src = reinterpret_cast<const float4*>(a.rec) + (size_t)g * stride4;
#pragma unroll
        for (int k = 0; k < R4; ++k) r[k] = __ldg(src + k);
      } else {
#pragma unroll
        for (int k = 0; k < R4; ++k) r[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    // N <= 6: the records of chunk i + 1 are loaded into registers while
    // chunk i is built; larger records are loaded right after a build (the
    // latency overlaps the next stage wait) to keep the register count down.
    constexpr bool PRE = N <= 6;
    float4 cur[R4], nxt[PRE ? R4 : 1];
    load(cand(0), cur);
    int g_next = cand(1);
    for (int i = 0; i < nchunks; ++i) {
      const int s = i % CS;
      if constexpr (PRE) {
        load(g_next, nxt);  // chunk i + 1 (zeros past the end)
        g_next = cand(i + 2);
      }
      bool ok = true;
      if (i >= CS) ok = warp_wait(&coef_empty[s], ((i / CS) - 1) & 1, abort_flag);
      if (!ok && lane == 0) fail();
      uint8_t* st = Cst + s * S::C_STAGE;
      bool scaled = false;
      if (ok) {
        float buf[R];
#pragma unroll
        for (int k = 0; k < R4; ++k) {
          buf[4 * k] = cur[k].x; buf[4 * k + 1] = cur[k].y;
          buf[4 * k + 2] = cur[k].z; buf[4 * k + 3] = cur[k].w;
        }
        float mt[N], tA[N];
#pragma unroll
        for (int d = 0; d < N; ++d) mt[d] = buf[P + d] - sctr[d];
        float cst = 0.0f;
#pragma unroll
        for (int d = 0; d < N; ++d) {
          float s2 = 0.0f;
#pragma unroll
          for (int k = 0; k < N; ++k) s2 = fmaf(buf[d >= k ? tri(d) + k : tri(k) + d], mt[k], s2);
          tA[d] = s2;
          cst = fmaf(mt[d], s2, cst);
        }
        // coefficients kb .. kb + 7 (kb compile-time after unrolling):
        // quadratic (d, e), linear d, constant, zero padding
        auto cblock = [&](int kb, float (&v)[8]) {
#pragma unroll
          for (int q = 0; q < 8; ++q) v[q] = 0.0f;
#pragma unroll
          for (int d = 0; d < N; ++d)
#pragma unroll
            for (int e2 = 0; e2 <= d; ++e2) {
              const int p = tri(d) + e2;
              if (p >= kb && p < kb + 8)
                v[p - kb] = kNegHalfLog2eH * (d == e2 ? buf[p] : 2.0f * buf[p]) * (hsc[d] * hsc[e2]);
            }
#pragma unroll
          for (int d = 0; d < N; ++d)
            if (P + d >= kb && P + d < kb + 8) v[P + d - kb] = (kNegHalfLog2eH * -2.0f) * tA[d] * hsc[d];
          if (P + N >= kb && P + N < kb + 8) v[P + N - kb] = kNegHalfLog2eH * cst;
        };
        float mx = 0.0f;
#pragma unroll
        for (int kb = 0; kb < KP; kb += 8) {
          float v[8];
          cblock(kb, v);
#pragma unroll
          for (int q = 0; q < 8; ++q) mx = fmaxf(mx, fabsf(v[q]));
        }
        float back = 1.0f, down = 1.0f;
        if (mx > kRowMax) {  // divide the row by 2^e, e = exponent(mx) - 13
          int e = (int)((__float_as_uint(mx) >> 23) & 0xffu) - 127 - 13;
          e = e > 120 ? 120 : e;
          down = __uint_as_float((uint32_t)(127 - e) << 23);
          back = __uint_as_float((uint32_t)(127 + e) << 23);
          scaled = true;
        }
#pragma unroll
        for (int kb = 0; kb < KP; kb += 8) {
          float v[8];
          cblock(kb, v);
          uint4 h, l;
          split_h2(v[0] * down, v[1] * down, h.x, l.x);
          split_h2(v[2] * down, v[3] * down, h.y, l.y);
          split_h2(v[4] * down, v[5] * down, h.z, l.z);
          split_h2(v[6] * down, v[7] * down, h.w, l.w);
          const uint32_t off = kmajor_off_h(j, kb, S::SBO);
          *reinterpret_cast<uint4*>(st + off) = h;
          *reinterpret_cast<uint4*>(st + S::B_BYTES + off) = l;
        }
        float* wd = reinterpret_cast<float*>(st + 2 * S::B_BYTES) + (j >> 1) * 8 + (j & 1);
        wd[0] = buf[P + N];
        wd[2] = buf[P + N + 1];
        wd[4] = buf[P + N + 2];
        wd[6] = back;
      }
      const bool any_scaled = __any_sync(0xffffffffu, scaled);
      if (lane == 0) sflag[s][warp] = any_scaled ? 1 : 0;
      fence_proxy_async();
      warp_arrive(&coef_full[s]);
      if constexpr (PRE) {
#pragma unroll
        for (int k = 0; k < R4; ++k) cur[k] = nxt[k];
      }
      // one decision per warp
      if (__shfl_sync(0xffffffffu, (!ok || *abort_flag) ? 1 : 0, 0)) break;
      if constexpr (!PRE) {
        load(g_next, cur);  // chunk i + 1
        g_next = cand(i + 2);
      }
    }
  } else if (warp == 12) {
    // ---- MMA issuer
    if (lane == 0) {
      // descriptor bases (a descriptor for base + off is base + off / 16)
      const uint64_t dA0 = smem_desc(smem_u32(Ahi), 128, S::SBO);
      const uint64_t dB0 = smem_desc(smem_u32(Cst), 128, S::SBO);
      constexpr uint64_t A_LO = S::PHI_BYTES >> 4, B_LO = S::B_BYTES >> 4;
      constexpr uint32_t IDESC = idesc_f16(NC);
      for (int i = 0; i < nchunks; ++i) {
        const int s = i % CS, b = i & 1;
        bool ok = mbar_wait_sleep(&coef_full[s], (i / CS) & 1, abort_flag);
        const uint64_t dbh = dB0 + (uint64_t)((s * S::C_STAGE) >> 4);
        for (int h = 0; ok && h < nh; ++h) {
          // row block h of buffer b is free once its epilogue group has read chunk i - 2
          if (i >= 2) ok = mbar_wait_sleep(&acc_empty[2 * b + h], ((i >> 1) - 1) & 1, abort_flag);
          if (!ok) break;
          fence_after_sync();
          const uint32_t d = tmem + (uint32_t)(b * 256 + h * 128);
          const uint64_t dah = dA0 + (uint64_t)((h * S::HALF_BYTES) >> 4);
#pragma unroll
          for (int ks = 0; ks < KP / 16; ++ks) {
            const uint64_t ko = (uint64_t)ks * 16u;  // two 16-byte core matrices per K step
            mma_f16(d, dah + ko, dbh + ko, IDESC, ks > 0 ? 1u : 0u);
            mma_f16(d, dah + ko, dbh + B_LO + ko, IDESC, 1u);
            mma_f16(d, dah + A_LO + ko, dbh + ko, IDESC, 1u);
          }
          mma_commit(&acc_full[2 * b + h]);
        }
        if (!ok) {
          fail();
          break;
        }
        mma_commit(&coef_empty[s]);
      }
    }
  } else {
    // ---- epilogue (tcgen05.ld 16x256b: thread t holds lanes t/4 and t/4 + 8
    // of a 16-lane half at columns 2 (t % 4) + {0, 1} of every 8-column group,
    // so each weight load serves four query rows)
    const int quad = warp & 3, h = (warp - 4) >> 2;
    const int tq = lane & 3, tr = lane >> 2;
    // rows ri = hb * 2 + r8: 16-lane half hb, lane t/4 + 8 r8; .x / .y
    // accumulate the even / odd column of the thread's pairs
    float2 acc[4][3];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[r][c] = make_float2(0.f, 0.f);
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(h * 128);
    // 32-column block n of buffer b: both 16-lane halves
    auto load = [&](int b, int n, uint32_t (&v)[2][16]) {
#pragma unroll
      for (int hb = 0; hb < 2; ++hb)
        tmem_ld16x256_x4_nowait(lane_base + ((uint32_t)(hb * 16) << 16) + (uint32_t)(b * 256 + n * 32),
                                v[hb]);
    };
    // accumulate block n (columns 32 n + 8 k + 2 tq + {0, 1}, k = 0..3): the
    // 32 exponentials first, in place (independent MUFU operations whose
    // latency overlaps), then the colour sums
    auto use = [&](const float* wp, int n, uint32_t (&v)[2][16], auto sc_tag) {
      constexpr bool SC = decltype(sc_tag)::value;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float2 sc = make_float2(1.f, 1.f);
        if (SC) sc = *reinterpret_cast<const float2*>(wp + (16 * n + 4 * k) * 8 + 6);
#pragma unroll
        for (int hb = 0; hb < 2; ++hb)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float sv = __uint_as_float(v[hb][4 * k + j]);
            if (SC) sv *= (j & 1) ? sc.y : sc.x;
            v[hb][4 * k + j] = __float_as_uint(ex2_approx(sv));
          }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float* wk = wp + (16 * n + 4 * k) * 8;
        const float4 w01 = *reinterpret_cast<const float4*>(wk);
        const float2 w2 = *reinterpret_cast<const float2*>(wk + 4);
#pragma unroll
        for (int hb = 0; hb < 2; ++hb)
#pragma unroll
          for (int r8 = 0; r8 < 2; ++r8) {
            const float2 e = make_float2(__uint_as_float(v[hb][4 * k + 2 * r8]),
                                         __uint_as_float(v[hb][4 * k + 2 * r8 + 1]));
            const int ri = hb * 2 + r8;
            acc[ri][0] = __ffma2_rn(make_float2(w01.x, w01.y), e, acc[ri][0]);
            acc[ri][1] = __ffma2_rn(make_float2(w01.z, w01.w), e, acc[ri][1]);
            acc[ri][2] = __ffma2_rn(w2, e, acc[ri][2]);
          }
      }
    };
    // one chunk: four 32-column blocks, block n + 1 loading while block n is used
    auto chunk = [&](int b, const float* wp, auto sc_tag) {
      uint32_t va[2][16], vb[2][16];
      load(b, 0, va);
      tmem_wait_ld();
      tmem_reg_fence16(va[0]);
      tmem_reg_fence16(va[1]);
      load(b, 1, vb);
      use(wp, 0, va, sc_tag);
      tmem_wait_ld();
      tmem_reg_fence16(vb[0]);
      tmem_reg_fence16(vb[1]);
      load(b, 2, va);
      use(wp, 1, vb, sc_tag);
      tmem_wait_ld();
      tmem_reg_fence16(va[0]);
      tmem_reg_fence16(va[1]);
      load(b, 3, vb);
      use(wp, 2, va, sc_tag);
      tmem_wait_ld();
      tmem_reg_fence16(vb[0]);
      tmem_reg_fence16(vb[1]);
      // this warp's reads of buffer b are complete
      fence_before_sync();
      warp_arrive(&acc_empty[2 * b + h]);
      use(wp, 3, vb, sc_tag);
    };
    const bool my_block = h < nh;
    for (int i = 0; my_block && i < nchunks; ++i) {
      const int s = i % CS, b = i & 1;
      bool ok = warp_wait(&acc_full[2 * b + h], (i >> 1) & 1, abort_flag);
      if (ok) ok = warp_wait(&coef_full[s], (i / CS) & 1, abort_flag);
      if (!ok) {
        if (lane == 0) fail();
        break;
      }
      fence_after_sync();
      const int4 fl = *reinterpret_cast<const int4*>(&sflag[s][0]);
      const bool scaled = (fl.x | fl.y | fl.z | fl.w) != 0;
      // weight pair entries of this thread: p = 16 n + 4 k + tq
      const float* wp = reinterpret_cast<const float*>(Cst + s * S::C_STAGE + 2 * S::B_BYTES) + tq * 8;
      if (scaled) chunk(b, wp, BoolTag<true>{});
      else chunk(b, wp, BoolTag<false>{});
      warp_arrive(&coef_empty[s]);
    }
    // ---- row sums over the pair halves and the four threads sharing a lane
    // (shuffles); thread tq writes row ri = tq
    if (my_block && !*abort_flag) {
#pragma unroll
      for (int ri = 0; ri < 4; ++ri) {
        float rs[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float v = acc[ri][c].x + acc[ri][c].y;
          v += __shfl_xor_sync(0xffffffffu, v, 1);
          v += __shfl_xor_sync(0xffffffffu, v, 2);
          rs[c] = v;
        }
        const int qr = h * 128 + quad * 32 + (ri >> 1) * 16 + (ri & 1) * 8 + tr;
        if (ri == tq && qr < nq) {
#pragma unroll
          for (int c = 0; c < 3; ++c) a.y[(qt + qr) * 3 + c] = rs[c];
        }
      }
    }
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
}

}  // namespace ndg
