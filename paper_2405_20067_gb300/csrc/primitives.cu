// primitives.cu -- scan, stable radix sort and bin boundaries used by the
// cull (bucket sort of Gaussians) and by the backward pass (transposing the
// tile-major candidate lists to Gaussian-major order without atomics).
#include "common.cuh"
#include "internal.h"

namespace ndg {

// ---- exclusive scan -------------------------------------------------------
constexpr int SC_THREADS = 1024;
constexpr int SC_ITEMS = 4;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

__device__ __forceinline__ long long warp_incl_scan(long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the total.
__device__ long long block_excl_scan(long long v, long long* out_excl) {
  __shared__ long long wsum[32];
  __shared__ long long wtotal;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  long long incl = warp_incl_scan(v);
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    long long s = lane < nw ? wsum[lane] : 0;
    long long si = warp_incl_scan(s);
    if (lane < nw) wsum[lane] = si - s;
    if (lane == 31) wtotal = si;  // nw <= 32
  }
  __syncthreads();
  *out_excl = incl - v + wsum[warp];
  long long total = wtotal;
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(SC_THREADS) scan_tiles(const long long* in, long long* out,
                                                         long long n, long long* bsum) {
  long long base = (long long)blockIdx.x * SC_TILE + (long long)threadIdx.x * SC_ITEMS;
  long long v[SC_ITEMS], s = 0;
#pragma unroll
  for (int i = 0; i < SC_ITEMS; ++i) {
    v[i] = base + i < n ? in[base + i] : 0;
    s += v[i];
  }
  long long ex;
  long long total = block_excl_scan(s, &ex);
#pragma unroll
  for (int i = 0; i < SC_ITEMS; ++i) {
    if (base + i < n) out[base + i] = ex;
    ex += v[i];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// One block scans the block sums in place (exclusive) and writes the total.
__global__ void __launch_bounds__(SC_THREADS) scan_sums(long long* bsum, long long nb,
                                                        long long* total_out) {
  long long carry = 0;
  for (long long c = 0; c < nb; c += SC_THREADS) {
    long long i = c + threadIdx.x;
    long long v = i < nb ? bsum[i] : 0, ex;
    long long t = block_excl_scan(v, &ex);
    if (i < nb) bsum[i] = ex + carry;
    carry += t;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void __launch_bounds__(SC_THREADS) scan_add(long long* out, long long n,
                                                       const long long* bsum) {
  long long base = (long long)blockIdx.x * SC_TILE + (long long)threadIdx.x * SC_ITEMS;
  long long add = bsum[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SC_ITEMS; ++i)
    if (base + i < n) out[base + i] += add;
}

size_t scan_temp_bytes(long long n) {
  long long nb = ceil_div<long long>(n > 0 ? n : 1, SC_TILE);
  return (size_t)(nb + 1) * sizeof(long long);
}

int scan_exclusive_i64(const long long* in, long long* out, long long n, void* temp,
                       cudaStream_t s) {
  long long nb = ceil_div<long long>(n > 0 ? n : 1, SC_TILE);
  long long* bsum = (long long*)temp;
  scan_tiles<<<(unsigned)nb, SC_THREADS, 0, s>>>(in, out, n, bsum);
  scan_sums<<<1, SC_THREADS, 0, s>>>(bsum, nb, out + n);
  if (nb > 1) {
    scan_add<<<(unsigned)nb, SC_THREADS, 0, s>>>(out, n, bsum);
    return 3;
  }
  return 2;
}

// ---- stable LSD radix sort, 8 bits per pass -------------------------------
// Tiles of RS_TILE keys per block; inside a block each warp owns a contiguous
// run of 32 * RS_ITEMS keys (lane l holds keys j * 32 + l).  Ranks keep the
// input order among equal digits: warp-level multisplit (match_any) in the
// order (j, lane) with warp-private digit histograms, an exclusive prefix over
// the warps of the block, then the block's global digit offsets from the scan
// of all (digit, block) counts.  Keys are reordered in shared memory first so
// that every digit's run is written to global memory contiguously.
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__device__ __forceinline__ long long rs_count(long long n_cap, const long long* n_dev) {
  if (!n_dev) return n_cap;
  long long n = *n_dev;
  return n < n_cap ? (n < 0 ? 0 : n) : n_cap;
}

__global__ void __launch_bounds__(RS_THREADS) rs_hist(const uint32_t* __restrict__ keys,
                                                      long long n_cap, const long long* n_dev,
                                                      int shift, long long* __restrict__ counts,
                                                      int nblocks) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const long long n = rs_count(n_cap, n_dev);
  const long long base = (long long)blockIdx.x * RS_TILE;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    const long long i = base + (long long)warp * 32 * RS_ITEMS + j * 32 + lane;
    const bool valid = i < n;
    const int d = valid ? (int)((keys[i] >> shift) & 255u) : 256 + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (valid && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&h[d], __popc(peers));
  }
  __syncthreads();
  counts[(long long)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS) rs_scatter(const uint32_t* __restrict__ kin,
                                                         const int32_t* __restrict__ vin,
                                                         uint32_t* __restrict__ kout,
                                                         int32_t* __restrict__ vout,
                                                         long long n_cap, const long long* n_dev,
                                                         int shift, const long long* __restrict__ offs,
                                                         int nblocks) {
  __shared__ int wh[RS_WARPS][256];   // per-warp digit counts, then per-warp exclusive prefix
  __shared__ int bstart[257];         // block-local start of each digit
  __shared__ long long goff[256];     // global offset of each digit for this block
  __shared__ uint32_t sk[RS_TILE];
  __shared__ int32_t sv[RS_TILE];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long n = rs_count(n_cap, n_dev);
  const long long base = (long long)blockIdx.x * RS_TILE;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) wh[w][tid] = 0;
  goff[tid] = offs[(long long)tid * nblocks + blockIdx.x];
  __syncthreads();
  uint32_t key[RS_ITEMS];
  int32_t val[RS_ITEMS];
  int dig[RS_ITEMS], rank[RS_ITEMS];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    const long long i = base + (long long)warp * 32 * RS_ITEMS + j * 32 + lane;
    const bool valid = i < n;
    key[j] = valid ? kin[i] : 0u;
    val[j] = valid ? (vin ? vin[i] : (int32_t)i) : 0;
    const int d = valid ? (int)((key[j] >> shift) & 255u) : 256 + lane;
    dig[j] = d;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    int before = 0;
    if (valid) before = wh[warp][d];
    __syncwarp();
    rank[j] = before + __popc(peers & lt);
    if (valid && (peers & lt) == 0) wh[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // exclusive prefix over warps (per digit) and block-local digit starts
  {
    int run = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      const int c = wh[w][tid];
      wh[w][tid] = run;
      run += c;
    }
    // run = block total of digit tid; exclusive scan over digits
    int incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    __shared__ int wsum[RS_WARPS];
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int off = 0;
    for (int w = 0; w < warp; ++w) off += wsum[w];
    bstart[tid] = incl - run + off;
    if (tid == RS_THREADS - 1) bstart[256] = incl + off;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    const int d = dig[j];
    if (d < 256) {
      const int p = bstart[d] + wh[warp][d] + rank[j];
      sk[p] = key[j];
      sv[p] = val[j];
    }
  }
  __syncthreads();
  const int nvalid = bstart[256];
  for (int p = tid; p < nvalid; p += RS_THREADS) {
    const uint32_t k = sk[p];
    const int d = (int)((k >> shift) & 255u);
    const long long g = goff[d] + (p - bstart[d]);
    kout[g] = k;
    vout[g] = sv[p];
  }
}

size_t radix_temp_bytes(long long n_cap) {
  long long nb = ceil_div<long long>(n_cap > 0 ? n_cap : 1, RS_TILE);
  size_t counts = (size_t)(256 * nb + 1) * sizeof(long long);
  counts = (counts + 255) / 256 * 256;
  return 2 * counts + scan_temp_bytes(256 * nb);
}

int radix_sort_pairs(const uint32_t* keys_in, const int32_t* vals_in, uint32_t* keys_a,
                      int32_t* vals_a, uint32_t* keys_b, int32_t* vals_b, long long n_cap,
                      const long long* n_dev, int bits, void* temp, cudaStream_t s,
                      uint32_t** keys_out, int32_t** vals_out) {
  long long nb = ceil_div<long long>(n_cap > 0 ? n_cap : 1, RS_TILE);
  size_t counts_b = ((size_t)(256 * nb + 1) * sizeof(long long) + 255) / 256 * 256;
  long long* counts = (long long*)temp;
  long long* offs = (long long*)((char*)temp + counts_b);
  void* stemp = (char*)temp + 2 * counts_b;
  const int passes = bits < 1 ? 1 : (bits + 7) / 8;
  uint32_t* kbuf[2] = {keys_a, keys_b};
  int32_t* vbuf[2] = {vals_a, vals_b};
  int launched = 0;
  for (int p = 0; p < passes; ++p) {
    // pass p reads buffer p & 1 (the caller's input on pass 0) and writes the other
    const uint32_t* ksrc = p == 0 ? keys_in : kbuf[p & 1];
    const int32_t* vsrc = p == 0 ? vals_in : vbuf[p & 1];
    const int dst = (p + 1) & 1;
    rs_hist<<<(unsigned)nb, RS_THREADS, 0, s>>>(ksrc, n_cap, n_dev, 8 * p, counts, (int)nb);
    launched += 2 + scan_exclusive_i64(counts, offs, 256 * nb, stemp, s);
    rs_scatter<<<(unsigned)nb, RS_THREADS, 0, s>>>(ksrc, vsrc, kbuf[dst], vbuf[dst], n_cap, n_dev,
                                                   8 * p, offs, (int)nb);
  }
  *keys_out = kbuf[passes & 1];
  *vals_out = vbuf[passes & 1];
  return launched;
}

// ---- boundaries of sorted bins --------------------------------------------
__global__ void bin_bounds_kernel(const uint32_t* sorted, long long n_cap, const long long* n_dev,
                                  int nbins, long long* off) {
  const long long n = rs_count(n_cap, n_dev);
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  long long prev = i == 0 ? -1 : (long long)min((uint32_t)nbins, sorted[i - 1]);
  long long cur = i == n ? nbins : (long long)min((uint32_t)nbins, sorted[i]);
  for (long long b = prev + 1; b <= cur; ++b) off[b] = i;
}

int bin_boundaries(const uint32_t* sorted, long long n_cap, const long long* n_dev, int nbins,
                   long long* off, cudaStream_t s) {
  long long threads = n_cap + 1;
  bin_bounds_kernel<<<(unsigned)ceil_div<long long>(threads, 256), 256, 0, s>>>(sorted, n_cap, n_dev,
                                                                             nbins, off);
  return 1;
}

// ---- Gaussian-major order of candidate entries -------------------------------
// A stable counting sort of the entries by id, using that an id occurs at
// most once per tile (so the stable order of an id's entries is their tile
// order): per-id counts (atomics), exclusive scan (goff), scatter of
// (tile, entry) through per-id cursors (atomics: arbitrary order inside a
// segment), then per segment (one warp) a bitmap of its tiles in shared
// memory: an entry's rank is the number of set bits below its tile.
__global__ void tr_count(const int32_t* __restrict__ ids, long long n_cap,
                         const long long* __restrict__ n_dev, int nid,
                         unsigned long long* __restrict__ cnt) {
  const long long n = rs_count(n_cap, n_dev);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int g = ids[e];
    if ((unsigned)g < (unsigned)nid) atomicAdd(cnt + g, 1ull);
  }
}

// One block per tile: its entries [offsets[t], offsets[t+1]).
__global__ void __launch_bounds__(256) tr_scatter(const long long* __restrict__ offsets,
                                                  const int32_t* __restrict__ ids, int nid,
                                                  unsigned long long* __restrict__ cur,
                                                  unsigned long long* __restrict__ te) {
  const long long t = blockIdx.x;
  const long long b = offsets[t], en = offsets[t + 1];
  // four entries per thread in flight (independent cursor atomics); the
  // slot order inside a segment is not used (tr_rank ranks by tile)
  long long e = b + threadIdx.x;
  for (; e + 3 * (long long)blockDim.x < en; e += 4 * (long long)blockDim.x) {
    int g[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) g[u] = ids[e + u * (long long)blockDim.x];
    unsigned long long slot[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      slot[u] = (unsigned)g[u] < (unsigned)nid ? atomicAdd(cur + g[u], 1ull) : ~0ull;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (slot[u] != ~0ull)
        te[slot[u]] = ((unsigned long long)t << 32) | (unsigned long long)(e + u * (long long)blockDim.x);
  }
  for (; e < en; e += blockDim.x) {
    const int g = ids[e];
    if ((unsigned)g < (unsigned)nid)
      te[atomicAdd(cur + g, 1ull)] = ((unsigned long long)t << 32) | (unsigned long long)e;
  }
}

// One warp per segment (persistent over segments); words = ceil(T / 32).
__global__ void __launch_bounds__(256) tr_rank(const long long* __restrict__ goff, int nid,
                                               const unsigned long long* __restrict__ te,
                                               int words, int32_t* __restrict__ perm) {
  extern __shared__ uint32_t tsm[];  // per warp: bitmap [words], prefix [words]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* bm = tsm + (size_t)warp * 2 * words;
  uint32_t* pre = bm + words;
  for (int g = blockIdx.x * 8 + warp; g < nid; g += gridDim.x * 8) {
    const long long b = goff[g];
    const int L = (int)(goff[g + 1] - b);
    if (L == 0) continue;
    if (L == 1) {
      if (lane == 0) perm[b] = (int32_t)(te[b] & 0xffffffffull);
      continue;
    }
    // tile span of the segment: only those bitmap words are touched
    for (int w = lane; w < words; w += 32) bm[w] = 0u;
    __syncwarp();
    for (int i = lane; i < L; i += 32) {
      const uint32_t t = (uint32_t)(te[b + i] >> 32);
      atomicOr(bm + (t >> 5), 1u << (t & 31));
    }
    __syncwarp();
    // exclusive prefix of the words' popcounts (lane-sequential chunks + warp scan)
    const int per = (words + 31) / 32;
    int run = 0;
    for (int k = 0; k < per; ++k) {
      const int w = lane * per + k;
      if (w < words) run += __popc(bm[w]);
    }
    int incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    int acc = incl - run;
    for (int k = 0; k < per; ++k) {
      const int w = lane * per + k;
      if (w < words) {
        pre[w] = (uint32_t)acc;
        acc += __popc(bm[w]);
      }
    }
    __syncwarp();
    for (int i = lane; i < L; i += 32) {
      const unsigned long long v = te[b + i];
      const uint32_t t = (uint32_t)(v >> 32);
      const int r = (int)pre[t >> 5] + __popc(bm[t >> 5] & ((1u << (t & 31)) - 1u));
      perm[b + r] = (int32_t)(v & 0xffffffffull);
    }
    __syncwarp();
  }
}

size_t transpose_temp_bytes(int nid) {
  const size_t c = ((size_t)(nid > 0 ? nid : 1) * sizeof(unsigned long long) + 255) / 256 * 256;
  return c + scan_temp_bytes(nid > 0 ? nid : 1);
}

int transpose_entries(const int32_t* ids, const long long* offsets, long long T, long long n_cap,
                      const long long* n_dev, int nid, long long* goff, unsigned long long* te,
                      int32_t* perm, void* temp, cudaStream_t s) {
  const size_t c = ((size_t)(nid > 0 ? nid : 1) * sizeof(unsigned long long) + 255) / 256 * 256;
  unsigned long long* cnt = (unsigned long long*)temp;
  void* stemp = (char*)temp + c;
  cudaMemsetAsync(cnt, 0, (size_t)(nid > 0 ? nid : 1) * sizeof(unsigned long long), s);
  long long blocks = ceil_div<long long>(n_cap > 0 ? n_cap : 1, 256);
  if (blocks > 4 * 1024) blocks = 4 * 1024;
  tr_count<<<(unsigned)blocks, 256, 0, s>>>(ids, n_cap, n_dev, nid, cnt);
  int launched = 1 + scan_exclusive_i64((const long long*)cnt, goff, nid, stemp, s);
  // the counts become the cursors: cur[g] = goff[g]
  cudaMemcpyAsync(cnt, goff, (size_t)nid * sizeof(long long), cudaMemcpyDeviceToDevice, s);
  if (T > 0) {
    tr_scatter<<<(unsigned)T, 256, 0, s>>>(offsets, ids, nid, cnt, te);
    ++launched;
  }
  if (nid > 0) {
    const int words = (int)((T + 31) / 32 > 0 ? (T + 31) / 32 : 1);
    const size_t smem = (size_t)8 * 2 * words * sizeof(uint32_t);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(tr_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int rb = ceil_div(nid, 8) < 152 * 8 ? ceil_div(nid, 8) : 152 * 8;
    tr_rank<<<(unsigned)rb, 256, smem, s>>>(goff, nid, te, words, perm);
    ++launched;
  }
  return launched;
}

}  // namespace ndg
