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

namespace ndg {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false after `limit` unsuccessful polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Matrix descriptor: no swizzle; addresses and offsets in 16-byte units.
// lbo: byte distance between core matrices along K; sbo: along M / N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor for kind::tf32: F32 accumulator, TF32 A and B, both
// K-major (TF32 operands cannot be MN-major), M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ float tf32_hi(float v) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
  return __uint_as_float(h);
}

// Byte offset of element (row, k) in the K-major no-swizzle layout.
__device__ __forceinline__ uint32_t kmajor_off(int row, int k, uint32_t sbo) {
  return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 2) * 128u + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k & 3) * 4u;
}

// Writes one K-major row (KP values, multiple of 4) split into hi / lo.
template <int KP>
__device__ __forceinline__ void store_row_split(uint8_t* hi, uint8_t* lo, int row, uint32_t sbo,
                                                const float (&v)[KP]) {
#pragma unroll
  for (int k = 0; k < KP; k += 4) {
    float4 h, l;
    h.x = tf32_hi(v[k]); l.x = v[k] - h.x;
    h.y = tf32_hi(v[k + 1]); l.y = v[k + 1] - h.y;
    h.z = tf32_hi(v[k + 2]); l.z = v[k + 2] - h.z;
    h.w = tf32_hi(v[k + 3]); l.w = v[k + 3] - h.w;
    const uint32_t off = kmajor_off(row, k, sbo);
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) = l;
  }
}

constexpr float kNegHalfLog2eTC = -0.72134752044448170368f;
constexpr uint32_t kWaitLimit = 1u << 26;

}  // namespace

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
  static constexpr uint32_t SMEM_USED = 2 * A_BYTES + 2 * B_BYTES + NC * 16 + 128;
  // at most 512 / NC CTAs may share an SM's tensor memory: request enough
  // shared memory that no more than that many are resident
  static constexpr uint32_t SMEM_FLOOR = (228u * 1024u) / (512u / NC + 1) + 1024u;
  static constexpr uint32_t SMEM = SMEM_USED > SMEM_FLOOR ? SMEM_USED : SMEM_FLOOR;
};

template <int N>
__global__ void __launch_bounds__(128) fwd_tc_kernel(FwdArgs a) {
  using S = TcShape<N>;
  constexpr int P = S::P, KP = S::KP, NC = S::NC, R = rec_floats(N), R4 = R / 4;
  extern __shared__ __align__(128) uint8_t dsm[];
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm + 127) & ~(uintptr_t)127);
  uint8_t* Ahi = base;
  uint8_t* Alo = Ahi + S::A_BYTES;
  uint8_t* Bhi = Alo + S::A_BYTES;
  uint8_t* Blo = Bhi + S::B_BYTES;
  float4* sw = reinterpret_cast<float4*>(Blo + S::B_BYTES);
  __shared__ uint64_t mbar;
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
    tmem_alloc(&tmem_base, NC < 32 ? 32 : NC);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&mbar, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t my_lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
  constexpr uint32_t IDESC = idesc_tf32(NC);

  float2 acc[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  const long long beg = a.offsets[t], end = a.offsets[t + 1];
  uint32_t phase = 0;
  for (long long c0 = beg; c0 < end; c0 += NC) {
    const int n = (int)(end - c0 < NC ? end - c0 : NC);
    // staging: coefficient rows of the chunk's candidates
    for (int j = tid; j < NC; j += 128) {
      const int g = j < n ? a.ids[c0 + j] : -1;
      float coef[KP];
      float4 wv = make_float4(0.f, 0.f, 0.f, 0.f);
      if ((unsigned)g < (unsigned)a.Ge) {
        const float4* src = reinterpret_cast<const float4*>(a.rec) + (size_t)g * R4;
        float buf[R];
#pragma unroll
        for (int i = 0; i < R4; ++i) {
          float4 v = __ldg(src + i);
          buf[4 * i] = v.x; buf[4 * i + 1] = v.y; buf[4 * i + 2] = v.z; buf[4 * i + 3] = v.w;
        }
        float mt[N], u[N];
#pragma unroll
        for (int i = 0; i < N; ++i) mt[i] = buf[P + i] - sctr[i];
        float cst = 0.0f;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          float s = 0.0f;
#pragma unroll
          for (int k = 0; k < N; ++k) s = fmaf(buf[i >= k ? tri(i) + k : tri(k) + i], mt[k], s);
          u[i] = s;
          cst = fmaf(mt[i], s, cst);
        }
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
          for (int k = 0; k <= i; ++k)
            coef[tri(i) + k] = kNegHalfLog2eTC * (i == k ? buf[tri(i) + k] : 2.0f * buf[tri(i) + k]);
#pragma unroll
        for (int i = 0; i < N; ++i) coef[P + i] = kNegHalfLog2eTC * (-2.0f * u[i]);
        coef[P + N] = kNegHalfLog2eTC * cst;
        wv = make_float4(buf[P + N], buf[P + N + 1], buf[P + N + 2], 0.0f);
      } else {
#pragma unroll
        for (int k = 0; k < P + N + 1; ++k) coef[k] = 0.0f;
      }
#pragma unroll
      for (int k = P + N + 1; k < KP; ++k) coef[k] = 0.0f;
      store_row_split<KP>(Bhi, Blo, j, S::SBO_B, coef);
      sw[j] = wv;
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
      for (int ks = 0; ks < KP / 8; ++ks) {
        const uint32_t ko = (uint32_t)ks * 256u;  // two core matrices per K step of 8
        const uint64_t dah = smem_desc(ah + ko, 128, S::SBO_A);
        const uint64_t dal = smem_desc(al + ko, 128, S::SBO_A);
        const uint64_t dbh = smem_desc(bh + ko, 128, S::SBO_B);
        const uint64_t dbl = smem_desc(bl + ko, 128, S::SBO_B);
        mma_tf32(tmem, dah, dbh, IDESC, ks > 0 ? 1u : 0u);
        mma_tf32(tmem, dah, dbl, IDESC, 1u);
        mma_tf32(tmem, dal, dbh, IDESC, 1u);
      }
      mma_commit(&mbar);
    }
    if (!mbar_wait_bounded(&mbar, phase, kWaitLimit)) {
      atomicExch(&s_abort, 1);
      if (a.status) set_status(a.status, NDG_ERR_TIMEOUT);
    }
    phase ^= 1u;
    fence_after_sync();
    __syncthreads();
    if (s_abort) break;
    // epilogue: row tid of S, NC columns
#pragma unroll 1
    for (int cb = 0; cb < NC; cb += 32) {
      float v[32];
      tmem_ld32(my_lane_addr + (uint32_t)cb, v);
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        const float2 e = make_float2(ex2_approx(v[j]), ex2_approx(v[j + 1]));
        const float4 w0 = sw[cb + j], w1 = sw[cb + j + 1];
        acc[0] = __ffma2_rn(make_float2(w0.x, w1.x), e, acc[0]);
        acc[1] = __ffma2_rn(make_float2(w0.y, w1.y), e, acc[1]);
        acc[2] = __ffma2_rn(make_float2(w0.z, w1.z), e, acc[2]);
      }
    }
    fence_before_sync();
    __syncthreads();
  }
  if (s_abort) {
    // let any MMA still in flight finish before TMEM is released
    mbar_wait_bounded(&mbar, phase, kWaitLimit);
  }
  if (active && !s_abort) {
#pragma unroll
    for (int c = 0; c < 3; ++c) a.y[(q0 + tid) * 3 + c] = acc[c].x + acc[c].y;
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tmem, NC < 32 ? 32 : NC);
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
  const long long blocks = T * ((a.tile + 127) / 128);
#define L_TC(n)                                                                              \
  {                                                                                          \
    cudaFuncSetAttribute(fwd_tc_kernel<n>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                         (int)TcShape<n>::SMEM);                                             \
    fwd_tc_kernel<n><<<(unsigned)blocks, 128, TcShape<n>::SMEM, s>>>(a);                     \
  }
  NDG_SWITCH_N(N, L_TC)
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
