// fwd_h.cu -- the tensor-core forward, one CTA per query tile
// (ndg_forward, NDG_MODE_TC); the tile itself is fwd_tile (fwd_h_tile.cuh).
#include "fwd_h_tile.cuh"

namespace ndg {

// One CTA per tile (a tile list selects a subset; surplus CTAs leave at once).
template <int N>
__global__ void __launch_bounds__(416, 1) fwd_h_kernel(FwdArgs a) {
  extern __shared__ __align__(128) uint8_t dsm[];
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm + 127) & ~(uintptr_t)127);
  __shared__ FwdHSync sy;
  if (a.tiles && (int)blockIdx.x >= *a.n_tiles) return;
  const long long t = a.tiles ? (long long)a.tiles[blockIdx.x] : (long long)blockIdx.x;
  if (threadIdx.x < 32) {
    tmem_alloc(&sy.tmem_base, 512);
    tmem_relinquish();
  }
  fwd_tile<N>(a, t, base, sy);
  if (threadIdx.x < 32) {
    fence_after_sync();
    tmem_dealloc(sy.tmem_base, 512);
  }
}

#define NDG_H_CASE(n, call) case n: call(n); break;

unsigned fwd_tc_smem(int N) {
#define SM_H(n) return FwdHShape<n>::SMEM;
  switch (N) {
    NDG_H_CASE(1, SM_H) NDG_H_CASE(2, SM_H) NDG_H_CASE(3, SM_H) NDG_H_CASE(4, SM_H)
    NDG_H_CASE(5, SM_H) NDG_H_CASE(6, SM_H) NDG_H_CASE(7, SM_H) NDG_H_CASE(8, SM_H)
    NDG_H_CASE(9, SM_H) NDG_H_CASE(10, SM_H) NDG_H_CASE(11, SM_H) NDG_H_CASE(12, SM_H)
    default: return 0;
  }
#undef SM_H
}

int launch_fwd_tc(int N, const FwdArgs& a, long long T, cudaStream_t s) {
  if (T <= 0) return 0;
#define L_H(n)                                                                          \
  {                                                                                     \
    cudaFuncSetAttribute(fwd_h_kernel<n>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                         (int)FwdHShape<n>::SMEM);                                      \
    fwd_h_kernel<n><<<(unsigned)T, 416, FwdHShape<n>::SMEM, s>>>(a);                    \
  }
  switch (N) {
    NDG_H_CASE(1, L_H) NDG_H_CASE(2, L_H) NDG_H_CASE(3, L_H) NDG_H_CASE(4, L_H)
    NDG_H_CASE(5, L_H) NDG_H_CASE(6, L_H) NDG_H_CASE(7, L_H) NDG_H_CASE(8, L_H)
    NDG_H_CASE(9, L_H) NDG_H_CASE(10, L_H) NDG_H_CASE(11, L_H) NDG_H_CASE(12, L_H)
    default: return 0;
  }
#undef L_H
  return 1;
}

}  // namespace ndg
