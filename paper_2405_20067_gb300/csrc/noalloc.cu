// noalloc.cu -- ndg_forward_noalloc: the mixture evaluation for callers that
// cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc (or any allocator)
// at all: a renderer plugin inside a host application whose allocator owns
// the whole device memory budget, a per-frame callback that cannot afford
// the implicit device synchronisation an allocation may cause, or a process
// whose device footprint must be fixed when the library loads.  They still
// own their inputs and outputs, but have nowhere to put the scratch that
// ndg_forward keeps in the caller's workspace.  This entry point keeps that
// scratch -- the prepared per-Gaussian records -- in one file-scope device
// array instead, so it needs no workspace and allocates nothing.
//
// The array is NDG_NOALLOC_SCRATCH_BYTES (16 MiB) and every GPU that loads
// the library holds it until the process exits.  All calls share it and it
// keeps the last call's records; every call rewrites the records it reads
// before reading them, so nothing has to start at zero.  Calls that overlap
// on the GPU (different streams, different host threads) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "kernels.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[NDG_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  Host code
// cannot use g_noalloc_scratch directly: on the host that name is only a
// stand-in.  The address is looked up once per device, the first time this
// entry point runs on it, and kept for the life of the process; a
// cudaDeviceReset reloads the module and invalidates it (callers that reset a
// device must not call this entry point on it afterwards).
ndg_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NDG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return NDG_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return NDG_OK;
}

}  // namespace

extern "C" ndg_status ndg_forward_noalloc(const ndg_mixture* mix, const ndg_queries* q,
                                          const ndg_cull* cull, float* y, ndg_stream stream) {
  using namespace ndg;
  // the same argument rules as ndg_forward (sizes, NULL and misaligned
  // pointers), except that the candidate count E_dev is not needed here
  ndg_status st;
  if ((st = check_mix(mix)) || (st = check_queries(q))) return st;
  if (q->Q > 0 && (!y || !aligned(y, 4))) return NDG_ERR_INVALID_ARG;
  if (!cull || !cull->offsets || !aligned(cull->offsets, 8) || cull->E_cap < 0 ||
      (cull->E_cap > 0 && (!cull->ids || !aligned(cull->ids, 4))))
    return NDG_ERR_INVALID_ARG;
  const long long Ge = (long long)mix->G * (mix->has_children ? 2 : 1);
  const size_t need = (size_t)Ge * rec_floats(mix->N) * sizeof(float);
  if (need > (size_t)NDG_NOALLOC_SCRATCH_BYTES) return NDG_ERR_SCRATCH_LIMIT;
  void* scratch = nullptr;
  st = scratch_address(&scratch);
  if (st != NDG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  PrepArgs pa{};
  pa.G = mix->G;
  pa.Ge = (int)Ge;
  pa.mean = mix->mean;
  pa.theta = mix->theta;
  pa.alpha_raw = mix->alpha_raw;
  pa.color_raw = mix->color_raw;
  pa.u_theta = mix->u_theta;
  pa.m_u = mix->m_u;
  pa.c_alpha_raw = mix->c_alpha_raw;
  pa.c_color_raw = mix->c_color_raw;
  pa.rec = (float*)scratch;
  pa.status = nullptr;
  FwdArgs fa{};
  fa.x = q->x;
  fa.Q = q->Q;
  fa.tile = q->tile_size;
  fa.offsets = cull->offsets;
  fa.ids = cull->ids;
  fa.rec = pa.rec;
  fa.Ge = pa.Ge;
  fa.y = y;
  // A launch failure of this call is an error that was not pending before
  // it.  An error left pending by an earlier, unrelated call is neither
  // reported as this call's nor cleared.
  const cudaError_t before = cudaPeekAtLastError();
  launch_prep(mix->N, pa, s);
  launch_fwd(mix->N, fa, (q->Q + q->tile_size - 1) / q->tile_size, s);
  const cudaError_t after = cudaPeekAtLastError();
  if (after != cudaSuccess && after != before) {
    (void)cudaGetLastError();  // this call's own launch error: reported here
    return NDG_ERR_CUDA;
  }
  return NDG_OK;
}
