// internal.h -- host-side launchers shared between the libndg translation
// units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "ndg.h"

namespace ndg {

// ---- host-side argument checks (api.cu), shared by every entry point ------
// Each returns NDG_OK or NDG_ERR_INVALID_ARG without touching the device:
// sizes in range, required pointers present and 4-byte aligned (FP32 data).
bool aligned(const void* p, size_t a);
ndg_status check_mix(const ndg_mixture* m);
ndg_status check_queries(const ndg_queries* q);
ndg_status check_cull_params(const ndg_cull_params* cp);
ndg_status check_cull(const ndg_cull* c);  // also requires E_dev

// ---- primitives (primitives.cu) ------------------------------------------
// Exclusive prefix sum of n int64 values: out[0..n], out[n] = total.
// Every launcher returns the number of kernels it launched.
size_t scan_temp_bytes(long long n);
int scan_exclusive_i64(const long long* in, long long* out, long long n, void* temp,
                        cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on the low `bits` key bits.
// The element count is n_cap, or min(*n_dev, n_cap) when n_dev is given
// (read on the device, so the call can sit in a CUDA graph).  The input
// (keys_in, vals_in) is only read; vals_in == NULL means values 0, 1, 2, ...
// Buffers a and b (n_cap elements each) are the ping-pong storage; the
// result is returned in (keys_out, vals_out), one of the two.
size_t radix_temp_bytes(long long n_cap);
int radix_sort_pairs(const uint32_t* keys_in, const int32_t* vals_in, uint32_t* keys_a,
                      int32_t* vals_a, uint32_t* keys_b, int32_t* vals_b, long long n_cap,
                      const long long* n_dev, int bits, void* temp, cudaStream_t s,
                      uint32_t** keys_out, int32_t** vals_out);

// off[b] = first position whose sorted key is >= b, for b in [0, nbins];
// keys >= nbins count as nbins.
int bin_boundaries(const uint32_t* sorted, long long n_cap, const long long* n_dev,
                    int nbins, long long* off, cudaStream_t s);

// Gaussian-major order of candidate entries: goff[0..nid] segment offsets
// and perm[goff[g] .. goff[g+1]) the entries with id g in ascending order
// (the stable order of a sort by id).  Every id must occur at most once per
// tile (offsets [T+1] delimit the tiles' entries); te [n_cap] is scratch for
// (tile, entry) pairs; tr_rank uses T / 4 bytes of shared memory per warp
// (T <= 32768: 64 KB per block).
size_t transpose_temp_bytes(int nid);
int transpose_entries(const int32_t* ids, const long long* offsets, long long T, long long n_cap,
                      const long long* n_dev, int nid, long long* goff, unsigned long long* te,
                      int32_t* perm, void* temp, cudaStream_t s);

}  // namespace ndg
