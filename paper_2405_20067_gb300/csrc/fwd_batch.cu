// fwd_batch.cu -- many frames' tensor-core forwards in one persistent launch
// (ndg_forward_batch); the tile itself is fwd_tile (fwd_h_tile.cuh).
#include "fwd_h_tile.cuh"

namespace ndg {

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long v;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
  return v;
}

// Persistent CTAs (one per SM) over the (frame, tile) work list of a batch
// of frames of any N <= 12: a CTA takes the next item with an atomic
// cursor, renders that tile with fwd_tile<N> of the item's frame (so a
// frame's outputs equal those of its own fwd_h_kernel launch), and the CTA
// that completes a frame's last tile stamps the frame's completion time.
// Tensor memory is allocated once per CTA and reused by every tile.
__global__ void __launch_bounds__(416, 1) fwd_h_batch_kernel(FwdBatchArgs b) {
  extern __shared__ __align__(128) uint8_t dsm[];
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm + 127) & ~(uintptr_t)127);
  __shared__ FwdHSync sy;
  __shared__ long long s_item;
  __shared__ int s_stop;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_stop = 0;
    if (b.stamps) atomicMin(&b.stamps[0], globaltimer_ns());
  }
  if (tid < 32) {
    tmem_alloc(&sy.tmem_base, 512);
    tmem_relinquish();
  }
  for (;;) {
    // s_item is rewritten only after the previous tile's closing barrier,
    // which every thread passes after reading it
    if (tid == 0) s_item = s_stop ? b.n_items : (long long)atomicAdd(b.cursor, 1ull);
    __syncthreads();
    const long long item = s_item;
    if (item >= b.n_items) break;
    int f = 0, hi = b.n_frames - 1;  // the frame whose item range holds item
    while (f < hi) {
      const int mid = (f + hi + 1) >> 1;
      if (b.tile_start[mid] <= item) f = mid;
      else hi = mid - 1;
    }
    const FwdArgs a = b.frames[f];
    const long long t = item - b.tile_start[f];
    switch (b.N[f]) {
      case 1: fwd_tile<1>(a, t, base, sy); break;
      case 2: fwd_tile<2>(a, t, base, sy); break;
      case 3: fwd_tile<3>(a, t, base, sy); break;
      case 4: fwd_tile<4>(a, t, base, sy); break;
      case 5: fwd_tile<5>(a, t, base, sy); break;
      case 6: fwd_tile<6>(a, t, base, sy); break;
      case 7: fwd_tile<7>(a, t, base, sy); break;
      case 8: fwd_tile<8>(a, t, base, sy); break;
      case 9: fwd_tile<9>(a, t, base, sy); break;
      case 10: fwd_tile<10>(a, t, base, sy); break;
      case 11: fwd_tile<11>(a, t, base, sy); break;
      case 12: fwd_tile<12>(a, t, base, sy); break;
      default: break;  // the host admits 1 <= N <= 12 only
    }
    if (tid == 0) {
      if (sy.s_abort) s_stop = 1;  // a timed-out wait: take no further items
      __threadfence();
      const unsigned long long nt = (unsigned long long)(b.tile_start[f + 1] - b.tile_start[f]);
      if (atomicAdd(&b.done[f], 1ull) + 1ull == nt && b.stamps) b.stamps[1 + f] = globaltimer_ns();
    }
  }
  if (tid < 32) {
    fence_after_sync();
    tmem_dealloc(sy.tmem_base, 512);
  }
}

int launch_fwd_tc_batch(const FwdBatchArgs& b, unsigned smem, int grid, cudaStream_t s) {
  if (b.n_items <= 0 || grid <= 0) return 0;
  cudaFuncSetAttribute(fwd_h_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  fwd_h_batch_kernel<<<(unsigned)grid, 416, smem, s>>>(b);
  return 1;
}

}  // namespace ndg
