// api.cu -- the C ABI declared in include/ndg.h: argument checks, the
// workspace layout and the launch sequence of every entry point.
//
// Workspace layout (256-byte aligned regions).  A common part that every
// call may use, followed by ONE of two call-specific parts that start at the
// same offset (calls sharing a workspace are ordered on one stream, and the
// call-specific parts only hold temporaries of the call that owns them):
//   common : header (status word), loss partial sums, prepared records
//            [2 G_cap][R], densify scratch (flag, rank, fresh: [G_cap] each),
//            the forward's tile lists of NDG_MODE_AUTO ([2 T + 2])
//   cull   : per-tile projection bounds and bucket keys, per-Gaussian bucket
//            keys and bins, the bin sort's buffers and offsets, per-tile
//            counts and their scan, sort / scan temporaries
//   bwd    : per-entry partial records [E_cap][RP], the transposition sort's
//            buffers, per-Gaussian offsets and sums, sort temporaries
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "kernels.h"

using namespace ndg;

namespace ndg {

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

ndg_status check_mix(const ndg_mixture* m) {
  if (!m) return NDG_ERR_INVALID_ARG;
  if (m->N < 1 || m->N > NDG_MAX_N || m->G < 0 || m->G_cap < m->G) return NDG_ERR_INVALID_ARG;
  if (m->G > (1 << 30)) return NDG_ERR_INVALID_ARG;
  if (m->G > 0) {
    const float* need[4] = {m->mean, m->theta, m->alpha_raw, m->color_raw};
    for (const float* p : need)
      if (!p || !aligned(p, 4)) return NDG_ERR_INVALID_ARG;
    if (m->has_children) {
      const float* ch[4] = {m->u_theta, m->m_u, m->c_alpha_raw, m->c_color_raw};
      for (const float* p : ch)
        if (!p || !aligned(p, 4)) return NDG_ERR_INVALID_ARG;
    }
  }
  return NDG_OK;
}

ndg_status check_queries(const ndg_queries* q) {
  if (!q || q->Q < 0 || q->tile_size < 1 || q->tile_size > NDG_MAX_TILE) return NDG_ERR_INVALID_ARG;
  if (q->Q > 0 && (!q->x || !aligned(q->x, 4))) return NDG_ERR_INVALID_ARG;
  return NDG_OK;
}

ndg_status check_cull_params(const ndg_cull_params* cp) {
  if (!cp || cp->k < 0 || cp->k > NDG_MAX_K) return NDG_ERR_INVALID_ARG;
  if (cp->k > 0 && !cp->proj) return NDG_ERR_INVALID_ARG;
  if (cp->buckets < 1 || cp->buckets > NDG_MAX_BUCKETS) return NDG_ERR_INVALID_ARG;
  if (!(cp->cutoff >= 0.0f) || !std::isfinite(cp->cutoff)) return NDG_ERR_INVALID_ARG;
  if (!(cp->cutoff > 0.0f) && !(cp->k_sigma >= 0.0f)) return NDG_ERR_INVALID_ARG;
  if (!(cp->child_k_min >= 0.0f) || !std::isfinite(cp->child_k_min)) return NDG_ERR_INVALID_ARG;
  return NDG_OK;
}

ndg_status check_cull(const ndg_cull* c) {
  if (!c || !c->offsets || !c->E_dev || c->E_cap < 0) return NDG_ERR_INVALID_ARG;
  if (c->E_cap > 0 && !c->ids) return NDG_ERR_INVALID_ARG;
  return NDG_OK;
}

}  // namespace ndg

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kLossParts = 512;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Region {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t r = off;
    off += align_up(bytes ? bytes : 1);
    return r;
  }
};

struct Sizes {
  int N = 0, G_cap = 0, Ge_cap = 0, tile = 1, k = 0, KP = 0, B = 1;
  long long Q = 0, T = 0, E_cap = 0;
};

struct CommonLayout {
  size_t header, rec, loss, dflag, drank, dfresh, tlist, end;
};
struct CullLayout {
  size_t tb, range, tkey, gkey, gkey_sorted, bin, bk_a, bv_a, bk_b, bv_b, binoff, counts, excl, masks,
      tmp, end;
};
struct BwdLayout {
  size_t part, sk_a, sv_a, sk_b, sv_b, goff, gsum, te, tmp, end;
};

CommonLayout common_layout(const Sizes& z) {
  Region r;
  CommonLayout c;
  c.header = r.take(sizeof(WsHeader));
  c.loss = r.take(kLossParts * sizeof(double));  // fixed offset: ndg_loss_l2 knows no sizes
  c.rec = r.take((size_t)z.Ge_cap * rec_tc_floats(z.N) * sizeof(float));
  c.dflag = r.take((size_t)z.G_cap * sizeof(int));
  c.drank = r.take((size_t)z.G_cap * sizeof(int));
  c.dfresh = r.take((size_t)z.G_cap * sizeof(int));
  // NDG_MODE_AUTO: the dense and sparse tile lists and their counts
  c.tlist = r.take(((size_t)2 * z.T + 2) * sizeof(int));
  c.end = r.off;
  return c;
}

long long mask_words(const Sizes& z) { return ((long long)z.Ge_cap + 31) / 32 + 8; }

CullLayout cull_layout(const Sizes& z, size_t base) {
  Region r;
  r.off = base;
  CullLayout c;
  const int nb = z.k > 0 ? z.B : 1;
  c.tb = r.take((size_t)z.T * z.k * 2 * sizeof(float));
  c.range = r.take(3 * NDG_MAX_K * sizeof(float));
  c.tkey = r.take((size_t)z.T * 2 * z.KP);
  c.gkey = r.take((size_t)z.Ge_cap * 2 * z.KP);
  c.gkey_sorted = r.take((size_t)z.Ge_cap * 2 * z.KP);
  c.bin = r.take((size_t)z.Ge_cap * 4);
  c.bk_a = r.take((size_t)z.Ge_cap * 4);
  c.bv_a = r.take((size_t)z.Ge_cap * 4);
  c.bk_b = r.take((size_t)z.Ge_cap * 4);
  c.bv_b = r.take((size_t)z.Ge_cap * 4);
  c.binoff = r.take(((size_t)nb * nb + 1) * sizeof(long long));
  // per (tile, warp slice) survivor counts and their exclusive scan
  c.counts = r.take((size_t)(8 * z.T + 1) * sizeof(long long));
  c.excl = r.take((size_t)(8 * z.T + 1) * sizeof(long long));
  // survivor ballots: a tile visits each Gaussian at most once
  c.masks = r.take((size_t)(z.T > 0 ? z.T : 1) * mask_words(z) * sizeof(uint32_t));
  size_t t1 = radix_temp_bytes(z.Ge_cap), t2 = scan_temp_bytes(8 * z.T + 1);
  c.tmp = r.take(t1 > t2 ? t1 : t2);
  c.end = r.off;
  return c;
}

// longest per-Gaussian segment (= tiles) the shared-memory segment sort takes
constexpr long long kMaxSegSort = 32768;

BwdLayout bwd_layout(const Sizes& z, size_t base) {
  Region r;
  r.off = base;
  BwdLayout b;
  b.part = r.take((size_t)z.E_cap * part_floats(z.N) * sizeof(float));
  b.sk_a = r.take((size_t)z.E_cap * 4);
  b.sv_a = r.take((size_t)z.E_cap * 4);
  b.sk_b = r.take((size_t)z.E_cap * 4);
  b.sv_b = r.take((size_t)z.E_cap * 4);
  b.goff = r.take(((size_t)z.Ge_cap + 1) * sizeof(long long));
  b.gsum = r.take((size_t)z.Ge_cap * part_floats(z.N) * sizeof(float));
  b.te = r.take((size_t)z.E_cap * sizeof(unsigned long long));
  {
    const size_t t1 = radix_temp_bytes(z.E_cap), t2 = transpose_temp_bytes(z.Ge_cap);
    b.tmp = r.take(t1 > t2 ? t1 : t2);
  }
  b.end = r.off;
  return b;
}

Sizes make_sizes(const ndg_mixture* m, const ndg_queries* q, const ndg_cull_params* cp,
                 long long E_cap) {
  Sizes z;
  z.N = m->N;
  z.G_cap = m->G_cap;
  z.Ge_cap = 2 * m->G_cap;
  z.Q = q ? q->Q : 0;
  z.tile = q ? q->tile_size : 1;
  z.T = q ? (z.Q + z.tile - 1) / z.tile : 0;
  z.k = cp ? cp->k : 0;
  z.KP = key_pad(z.k);
  z.B = cp ? cp->buckets : 1;
  z.E_cap = E_cap;
  return z;
}

int bits_for(long long n_values) {  // bits to hold values 0 .. n_values - 1
  int b = 1;
  while (b < 40 && (1ll << b) < n_values) ++b;
  return b;
}

ndg_status cuda_ok() {
  return cudaGetLastError() == cudaSuccess ? NDG_OK : NDG_ERR_CUDA;
}

__global__ void finalize_offsets_kernel(const long long* __restrict__ excl, long long T,
                                        long long E_cap, long long* __restrict__ offsets,
                                        long long* __restrict__ E_dev, int* status) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t > T) return;
  long long v = excl[8 * t];  // scanned per (tile, warp slice) counts
  offsets[t] = v < E_cap ? v : E_cap;
  if (t == T) {
    *E_dev = v;
    if (v > E_cap) set_status(status, NDG_ERR_CAPACITY);
  }
}

// Counts launches and records the trace events around the main kernel.
struct Tracer {
  ndg_trace* t;
  cudaStream_t s;
  long long n = 0;
  Tracer(ndg_trace* t_, cudaStream_t s_) : t(t_), s(s_) {}
  void begin() {
    if (t && t->main_begin) cudaEventRecord((cudaEvent_t)t->main_begin, s);
  }
  void end() {
    if (t && t->main_end) cudaEventRecord((cudaEvent_t)t->main_end, s);
  }
  Tracer& operator+=(int k) {
    n += k;
    return *this;
  }
  ~Tracer() {
    if (t) t->launches += n;
  }
};

PrepArgs prep_args(const ndg_mixture* m) {
  PrepArgs a{};
  a.G = m->G;
  a.Ge = m->has_children ? 2 * m->G : m->G;
  a.mean = m->mean;
  a.theta = m->theta;
  a.alpha_raw = m->alpha_raw;
  a.color_raw = m->color_raw;
  a.u_theta = m->u_theta;
  a.m_u = m->m_u;
  a.c_alpha_raw = m->c_alpha_raw;
  a.c_color_raw = m->c_color_raw;
  return a;
}

}  // namespace

extern "C" {

size_t ndg_workspace_size(const ndg_mixture* mix, const ndg_queries* q,
                          const ndg_cull_params* cp, long long E_cap) {
  if (!mix || mix->N < 1 || mix->N > NDG_MAX_N || mix->G_cap < 0) return 0;
  Sizes z = make_sizes(mix, q, cp, E_cap < 0 ? 0 : E_cap);
  CommonLayout c = common_layout(z);
  size_t need = c.end;
  if (cp) {
    CullLayout cl = cull_layout(z, c.end);
    need = cl.end > need ? cl.end : need;
  }
  if (E_cap > 0) {
    BwdLayout bl = bwd_layout(z, c.end);
    need = bl.end > need ? bl.end : need;
  }
  return need;
}

namespace {

// The cull (Section 3.2); xc != null: on position, for the Gaussians
// restricted to the constant inputs xc (ndg_build_cull_conditioned).
ndg_status build_cull(const ndg_mixture* mix, const ndg_queries* q, const ndg_cull_params* cp,
                      const float* xc, ndg_cull* out, void* ws, size_t ws_bytes,
                      ndg_stream stream, ndg_trace* trace) {
  ndg_status st;
  if ((st = check_mix(mix)) || (st = check_queries(q)) || (st = check_cull_params(cp)) ||
      (st = check_cull(out)))
    return st;
  if (xc && mix->N < 4) return NDG_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, kAlign)) return NDG_ERR_INVALID_ARG;
  Sizes z = make_sizes(mix, q, cp, out->E_cap);
  CommonLayout c = common_layout(z);
  CullLayout L = cull_layout(z, c.end);
  if (ws_bytes < L.end) return NDG_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  Tracer tr(trace, s);
  char* w = (char*)ws;
  int* status = &reinterpret_cast<WsHeader*>(w + c.header)->status;
  const int N = mix->N, k = cp->k, KP = z.KP, B = cp->buckets, nb = k > 0 ? B : 1;
  const long long T = z.T;
  float* tb = (float*)(w + L.tb);
  float* range = (float*)(w + L.range);
  uint8_t* tkey = (uint8_t*)(w + L.tkey);
  uint8_t* gkey = (uint8_t*)(w + L.gkey);
  if (k > 0) {
    tr += launch_tile_bounds(N, q->x, q->Q, q->tile_size, T, k, cp->proj, tb, s, xc ? 3 : N);
    tr += launch_cull_range(tb, T, k, B, q->Q, range, s);
    tr += launch_tile_keys(tb, T, k, KP, B, range, tkey, s);
  }
  PrepArgs pa = prep_args(mix);
  pa.k = k;
  pa.KP = KP;
  pa.B = B;
  pa.proj = cp->proj;
  pa.cutoff = cp->cutoff;
  pa.k_sigma = cp->k_sigma;
  pa.child_k_min = cp->child_k_min;
  pa.range = range;
  pa.gkey = k > 0 ? gkey : nullptr;
  pa.bin = (uint32_t*)(w + L.bin);
  pa.status = status;
  pa.xc = xc;
  // the records of every evaluation form (A, m, w, then M) as well, so that
  // an evaluation or backward of the same parameters may skip its own
  // preparation (NDG_RECORDS_READY)
  pa.rec = (float*)(w + c.rec);
  pa.rec_kind = 2;
  tr += launch_prep(N, pa, s);
  uint32_t* sk;
  int32_t* sv;
  tr += radix_sort_pairs((const uint32_t*)(w + L.bin), nullptr, (uint32_t*)(w + L.bk_a),
                   (int32_t*)(w + L.bv_a), (uint32_t*)(w + L.bk_b), (int32_t*)(w + L.bv_b), pa.Ge,
                   nullptr, bits_for((long long)nb * nb + 1), w + L.tmp, s, &sk, &sv);
  long long* binoff = (long long*)(w + L.binoff);
  tr += bin_boundaries(sk, pa.Ge, nullptr, nb * nb, binoff, s);
  uint8_t* gkey_sorted = (uint8_t*)(w + L.gkey_sorted);
  tr += launch_permute_keys(gkey, sv, pa.Ge, KP, gkey_sorted, s);
  CullTileArgs ca{};
  ca.tkey = tkey;
  ca.gkey = gkey_sorted;
  ca.binoff = binoff;
  ca.sorted_ids = sv;
  ca.B = B;
  ca.counts = (long long*)(w + L.counts);
  ca.excl = nullptr;
  ca.ids = nullptr;
  ca.E_cap = out->E_cap;
  ca.masks = (uint32_t*)(w + L.masks);
  ca.mask_words = mask_words(z);
  tr += launch_cull_tile(KP, ca, T, s);
  long long* excl = (long long*)(w + L.excl);
  tr += scan_exclusive_i64(ca.counts, excl, 8 * T, w + L.tmp, s);
  finalize_offsets_kernel<<<(unsigned)ceil_div<long long>(T + 1, 256), 256, 0, s>>>(
      excl, T, out->E_cap, out->offsets, out->E_dev, status);
  tr += 1;
  if (out->E_cap > 0) {
    ca.excl = excl;
    ca.ids = out->ids;
    tr.begin();
    tr += launch_cull_tile(KP, ca, T, s);
    tr.end();
  }
  return cuda_ok();
}

}  // namespace

ndg_status ndg_build_cull(const ndg_mixture* mix, const ndg_queries* q, const ndg_cull_params* cp,
                          ndg_cull* out, void* ws, size_t ws_bytes, ndg_stream stream,
                          ndg_trace* trace) {
  return build_cull(mix, q, cp, nullptr, out, ws, ws_bytes, stream, trace);
}

ndg_status ndg_build_cull_conditioned(const ndg_mixture* mix, const ndg_queries* q,
                                      const ndg_cull_params* cp, const float* xc, ndg_cull* out,
                                      void* ws, size_t ws_bytes, ndg_stream stream,
                                      ndg_trace* trace) {
  if (!xc) return NDG_ERR_INVALID_ARG;
  return build_cull(mix, q, cp, xc, out, ws, ws_bytes, stream, trace);
}

ndg_status ndg_forward(const ndg_mixture* mix, const ndg_queries* q, const ndg_cull* cull, int mode,
                       float* y, void* ws, size_t ws_bytes, ndg_stream stream,
                       ndg_trace* trace) {
  ndg_status st;
  const bool recs_ready = (mode & NDG_RECORDS_READY) != 0;
  mode &= ~NDG_RECORDS_READY;
  if ((st = check_mix(mix)) || (st = check_queries(q)) || (st = check_cull(cull))) return st;
  if (mode != NDG_MODE_FP32 && mode != NDG_MODE_TC && mode != NDG_MODE_AUTO)
    return NDG_ERR_INVALID_ARG;
  if (q->Q > 0 && !y) return NDG_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, kAlign)) return NDG_ERR_INVALID_ARG;
  Sizes z = make_sizes(mix, q, nullptr, 0);
  CommonLayout c = common_layout(z);
  if (ws_bytes < c.end) return NDG_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  Tracer tr(trace, s);
  char* w = (char*)ws;
  PrepArgs pa = prep_args(mix);
  pa.rec = (float*)(w + c.rec);
  // AUTO, or records left by ndg_build_cull: both A (tensor-core form) and
  // M (FP32 form) per record
  const bool kind2 = recs_ready || mode == NDG_MODE_AUTO;
  pa.rec_kind = kind2 ? 2 : (mode == NDG_MODE_TC ? 1 : 0);
  pa.status = &reinterpret_cast<WsHeader*>(w + c.header)->status;
  if (!recs_ready) tr += launch_prep(mix->N, pa, s);
  FwdArgs fa{};
  fa.x = q->x;
  fa.Q = q->Q;
  fa.tile = q->tile_size;
  fa.offsets = cull->offsets;
  fa.ids = cull->ids;
  fa.rec = pa.rec;
  fa.Ge = pa.Ge;
  fa.y = y;
  fa.status = pa.status;
  if (mode == NDG_MODE_AUTO) {
    // per tile: the tensor-core form where the candidate list makes the
    // contraction dense, the FP32 form elsewhere (the same kernels as the
    // two fixed modes, so each tile's outputs equal that mode's)
    int* lists = (int*)(w + c.tlist);
    int* n_dense = lists + 2 * z.T;
    cudaMemsetAsync(n_dense, 0, 2 * sizeof(int), s);
    tr += launch_tile_split(cull->offsets, z.T, NDG_AUTO_MIN_CANDIDATES(mix->N), lists, lists + z.T,
                            n_dense, n_dense + 1, s);
    FwdArgs ft = fa, ff = fa;
    ft.rec_stride4 = ff.rec_stride4 = rec_tc_floats(mix->N) / 4;
    ft.tiles = lists;
    ft.n_tiles = n_dense;
    ff.tiles = lists + z.T;
    ff.n_tiles = n_dense + 1;
    ff.mat_off4 = rec_floats(mix->N) / 4;
    tr.begin();
    tr += launch_fwd_tc(mix->N, ft, z.T, s);
    tr += launch_fwd(mix->N, ff, z.T, s);
    tr.end();
    return cuda_ok();
  }
  if (kind2) {
    fa.rec_stride4 = rec_tc_floats(mix->N) / 4;
    if (mode == NDG_MODE_FP32) fa.mat_off4 = rec_floats(mix->N) / 4;
  }
  tr.begin();
  tr += mode == NDG_MODE_TC ? launch_fwd_tc(mix->N, fa, z.T, s) : launch_fwd(mix->N, fa, z.T, s);
  tr.end();
  return cuda_ok();
}

namespace {

// ndg_forward_batch's descriptor workspace: the frames' forward arguments,
// their N, the item prefix over frames, per-frame completion counters and
// the work-list cursor (one host-to-device copy of a host image).
struct BatchLayout {
  size_t frames, N, tile_start, done, cursor, end;
};

BatchLayout batch_layout(int n) {
  BatchLayout b{};
  b.frames = 0;
  b.N = align_up(b.frames + (size_t)n * sizeof(FwdArgs));
  b.tile_start = align_up(b.N + (size_t)n * sizeof(int));
  b.done = align_up(b.tile_start + (size_t)(n + 1) * sizeof(long long));
  b.cursor = align_up(b.done + (size_t)n * sizeof(unsigned long long));
  b.end = align_up(b.cursor + sizeof(unsigned long long));
  return b;
}

}  // namespace

size_t ndg_batch_workspace_size(int n_frames) {
  return n_frames < 1 ? 0 : batch_layout(n_frames).end;
}

ndg_status ndg_forward_batch(const ndg_frame* frames, int n_frames, void* batch_ws,
                             size_t batch_ws_bytes, unsigned long long* stamps,
                             ndg_stream stream, ndg_trace* trace) {
  if (!frames || n_frames < 1 || n_frames > (1 << 24)) return NDG_ERR_INVALID_ARG;
  if (!batch_ws || !aligned(batch_ws, kAlign)) return NDG_ERR_INVALID_ARG;
  if (stamps && !aligned(stamps, 8)) return NDG_ERR_INVALID_ARG;
  const BatchLayout bl = batch_layout(n_frames);
  if (batch_ws_bytes < bl.end) return NDG_ERR_WORKSPACE;
  // every frame is checked before anything runs
  for (int f = 0; f < n_frames; ++f) {
    const ndg_frame& fr = frames[f];
    ndg_status st;
    if ((st = check_mix(fr.mix)) || (st = check_queries(fr.q)) || (st = check_cull(fr.cull)))
      return st;
    if (fr.q->Q > 0 && !fr.y) return NDG_ERR_INVALID_ARG;
    if (!fr.ws || !aligned(fr.ws, kAlign)) return NDG_ERR_INVALID_ARG;
    if (fr.ws_bytes < common_layout(make_sizes(fr.mix, fr.q, nullptr, 0)).end)
      return NDG_ERR_WORKSPACE;
    if (fr.flags & ~NDG_RECORDS_READY) return NDG_ERR_INVALID_ARG;
  }
  // one persistent CTA per SM (queried before anything is launched)
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return NDG_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Tracer tr(trace, s);
  std::vector<char> img(bl.end, 0);
  FwdArgs* fa = reinterpret_cast<FwdArgs*>(img.data() + bl.frames);
  int* Ns = reinterpret_cast<int*>(img.data() + bl.N);
  long long* ts = reinterpret_cast<long long*>(img.data() + bl.tile_start);
  long long items = 0;
  unsigned smem = 0;
  for (int f = 0; f < n_frames; ++f) {
    const ndg_frame& fr = frames[f];
    const Sizes z = make_sizes(fr.mix, fr.q, nullptr, 0);
    const CommonLayout c = common_layout(z);
    char* w = (char*)fr.ws;
    PrepArgs pa = prep_args(fr.mix);
    pa.rec = (float*)(w + c.rec);
    // the tensor-core form's records, or those of every form that the
    // frame's cull left there
    const bool ready = (fr.flags & NDG_RECORDS_READY) != 0;
    pa.rec_kind = ready ? 2 : 1;
    pa.status = &reinterpret_cast<WsHeader*>(w + c.header)->status;
    if (!ready) tr += launch_prep(fr.mix->N, pa, s);
    FwdArgs& a = fa[f];
    a.rec_stride4 = ready ? rec_tc_floats(fr.mix->N) / 4 : 0;
    a.x = fr.q->x;
    a.Q = fr.q->Q;
    a.tile = fr.q->tile_size;
    a.offsets = fr.cull->offsets;
    a.ids = fr.cull->ids;
    a.rec = pa.rec;
    a.Ge = pa.Ge;
    a.y = fr.y;
    a.status = pa.status;
    Ns[f] = fr.mix->N;
    ts[f] = items;
    if (fr.q->Q > 0) {
      items += z.T;
      const unsigned m = fwd_tc_smem(fr.mix->N);
      smem = m > smem ? m : smem;
    }
  }
  ts[n_frames] = items;
  char* bw = (char*)batch_ws;
  // pageable source: the copy has consumed img when the call returns
  cudaMemcpyAsync(bw, img.data(), bl.end, cudaMemcpyHostToDevice, s);
  if (stamps) {
    cudaMemsetAsync(stamps, 0, sizeof(unsigned long long) * (size_t)(n_frames + 1), s);
    cudaMemsetAsync(stamps, 0xff, sizeof(unsigned long long), s);  // start: min over CTAs
  }
  FwdBatchArgs b{};
  b.frames = reinterpret_cast<const FwdArgs*>(bw + bl.frames);
  b.N = reinterpret_cast<const int*>(bw + bl.N);
  b.tile_start = reinterpret_cast<const long long*>(bw + bl.tile_start);
  b.done = reinterpret_cast<unsigned long long*>(bw + bl.done);
  b.cursor = reinterpret_cast<unsigned long long*>(bw + bl.cursor);
  b.stamps = stamps;
  b.n_frames = n_frames;
  b.n_items = items;
  const int grid = (int)(items < (long long)sms ? items : (long long)sms);
  tr.begin();
  tr += launch_fwd_tc_batch(b, smem, grid, s);
  tr.end();
  return cuda_ok();
}

ndg_status ndg_loss_l2(long long Q, const float* y, const float* target, float* dy,
                       double* loss_dev, void* ws, size_t ws_bytes, ndg_stream stream,
                       ndg_trace* trace) {
  if (Q < 0 || !loss_dev || (Q > 0 && (!y || !target || !dy))) return NDG_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, kAlign)) return NDG_ERR_INVALID_ARG;
  const size_t off = align_up(sizeof(WsHeader));
  if (ws_bytes < off + kLossParts * sizeof(double)) return NDG_ERR_WORKSPACE;
  double* part = (double*)((char*)ws + off);
  Tracer tr(trace, (cudaStream_t)stream);
  tr.begin();
  tr += launch_loss(y, target, dy, 3 * Q, part, loss_dev, (cudaStream_t)stream);
  tr.end();
  return cuda_ok();
}

ndg_status ndg_loss_l2_shard(long long Q, long long Q_total, const float* y, const float* target,
                             float* dy, double* loss_dev, void* ws, size_t ws_bytes,
                             ndg_stream stream, ndg_trace* trace) {
  if (Q < 0 || Q_total < Q || !loss_dev || (Q > 0 && (!y || !target || !dy)))
    return NDG_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, kAlign)) return NDG_ERR_INVALID_ARG;
  const size_t off = align_up(sizeof(WsHeader));
  if (ws_bytes < off + kLossParts * sizeof(double)) return NDG_ERR_WORKSPACE;
  double* part = (double*)((char*)ws + off);
  Tracer tr(trace, (cudaStream_t)stream);
  tr.begin();
  tr += launch_loss(y, target, dy, 3 * Q, part, loss_dev, (cudaStream_t)stream, -1.0, 3 * Q_total);
  tr.end();
  return cuda_ok();
}

ndg_status ndg_loss_rel_l2(long long Q, const float* y, const float* target, float eps, float* dy,
                           double* loss_dev, void* ws, size_t ws_bytes, ndg_stream stream,
                           ndg_trace* trace) {
  if (Q < 0 || !loss_dev || (Q > 0 && (!y || !target || !dy))) return NDG_ERR_INVALID_ARG;
  if (!(eps > 0.0f) || !std::isfinite(eps)) return NDG_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, kAlign)) return NDG_ERR_INVALID_ARG;
  const size_t off = align_up(sizeof(WsHeader));
  if (ws_bytes < off + kLossParts * sizeof(double)) return NDG_ERR_WORKSPACE;
  double* part = (double*)((char*)ws + off);
  Tracer tr(trace, (cudaStream_t)stream);
  tr.begin();
  tr += launch_loss(y, target, dy, 3 * Q, part, loss_dev, (cudaStream_t)stream, (double)eps);
  tr.end();
  return cuda_ok();
}

ndg_status ndg_selftest_timeout(int which, void* ws, size_t ws_bytes, ndg_stream stream) {
  if (which != 0 && which != 1) return NDG_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, kAlign) || ws_bytes < sizeof(WsHeader)) return NDG_ERR_INVALID_ARG;
  launch_selftest_wait(&reinterpret_cast<WsHeader*>(ws)->status, which, (cudaStream_t)stream);
  return cuda_ok();
}

namespace {

// Gaussian-major order of the entries (the stable order of a sort by
// Gaussian index): the per-entry partial records are written in entry order
// and summed per Gaussian through this permutation.  A Gaussian occurs at
// most once per tile, so segments are at most T long: a counting sort with
// per-segment ranks by tile when T fits, else a radix sort.  launch = false
// only returns where the permutation is (the buffer depends on sizes alone).
int backward_order(const Sizes& z, const BwdLayout& L, const ndg_cull* cull, int Ge, char* w,
                   bool launch, cudaStream_t s, int32_t** sv_out) {
  long long* goff = (long long*)(w + L.goff);
  if (z.T <= kMaxSegSort) {
    *sv_out = (int32_t*)(w + L.sv_a);
    if (!launch) return 0;
    return transpose_entries(cull->ids, cull->offsets, z.T, cull->E_cap, cull->E_dev, Ge, goff,
                             (unsigned long long*)(w + L.te), *sv_out, w + L.tmp, s);
  }
  const int bits = bits_for(Ge > 0 ? Ge : 1);
  const int passes = bits < 1 ? 1 : (bits + 7) / 8;  // radix_sort_pairs: 8 bits a pass
  if (!launch) {
    *sv_out = (int32_t*)(w + ((passes & 1) ? L.sv_b : L.sv_a));
    return 0;
  }
  uint32_t* sk;
  int n = radix_sort_pairs((const uint32_t*)cull->ids, nullptr, (uint32_t*)(w + L.sk_a),
                           (int32_t*)(w + L.sv_a), (uint32_t*)(w + L.sk_b), (int32_t*)(w + L.sv_b),
                           cull->E_cap, cull->E_dev, bits, w + L.tmp, s, &sk, sv_out);
  n += bin_boundaries(sk, cull->E_cap, cull->E_dev, Ge, goff, s);
  return n;
}

ndg_status check_backward_args(const ndg_mixture* mix, const ndg_queries* q, const ndg_cull* cull,
                               void* ws, size_t ws_bytes) {
  ndg_status st;
  if ((st = check_mix(mix)) || (st = check_queries(q)) || (st = check_cull(cull))) return st;
  if (cull->E_cap >= (1ll << 31)) return NDG_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, kAlign)) return NDG_ERR_INVALID_ARG;
  const Sizes z = make_sizes(mix, q, nullptr, cull->E_cap);
  if (ws_bytes < bwd_layout(z, common_layout(z).end).end) return NDG_ERR_WORKSPACE;
  return NDG_OK;
}

}  // namespace

ndg_status ndg_backward_order(const ndg_mixture* mix, const ndg_queries* q, const ndg_cull* cull,
                              void* ws, size_t ws_bytes, ndg_stream stream, ndg_trace* trace) {
  ndg_status st;
  if ((st = check_backward_args(mix, q, cull, ws, ws_bytes))) return st;
  const Sizes z = make_sizes(mix, q, nullptr, cull->E_cap);
  const BwdLayout L = bwd_layout(z, common_layout(z).end);
  cudaStream_t s = (cudaStream_t)stream;
  Tracer tr(trace, s);
  int32_t* sv;
  tr.begin();
  tr += backward_order(z, L, cull, prep_args(mix).Ge, (char*)ws, true, s, &sv);
  tr.end();
  return cuda_ok();
}

ndg_status ndg_backward(const ndg_mixture* mix, const ndg_queries* q, const ndg_cull* cull,
                        int mode, const float* dy, ndg_mixture* grad, void* ws, size_t ws_bytes,
                        ndg_stream stream, ndg_trace* trace) {
  ndg_status st;
  const bool order_ready = (mode & NDG_BWD_ORDER_READY) != 0;
  const bool recs_ready = (mode & NDG_RECORDS_READY) != 0;
  mode &= ~(NDG_BWD_ORDER_READY | NDG_RECORDS_READY);
  if ((st = check_backward_args(mix, q, cull, ws, ws_bytes))) return st;
  if (mode == NDG_MODE_AUTO) mode = NDG_MODE_TC;
  if (mode != NDG_MODE_FP32 && mode != NDG_MODE_TC) return NDG_ERR_INVALID_ARG;
  if (!grad || grad->N != mix->N || grad->G != mix->G || grad->has_children != mix->has_children ||
      (st = check_mix(grad)))
    return st ? st : NDG_ERR_INVALID_ARG;
  if (q->Q > 0 && !dy) return NDG_ERR_INVALID_ARG;
  Sizes z = make_sizes(mix, q, nullptr, cull->E_cap);
  CommonLayout c = common_layout(z);
  BwdLayout L = bwd_layout(z, c.end);
  cudaStream_t s = (cudaStream_t)stream;
  Tracer tr(trace, s);
  char* w = (char*)ws;
  const int N = mix->N;
  PrepArgs pa = prep_args(mix);
  pa.rec = (float*)(w + c.rec);
  pa.rec_kind = mode == NDG_MODE_TC ? 2 : 0;
  pa.status = &reinterpret_cast<WsHeader*>(w + c.header)->status;
  // the tensor-core form reads the records ndg_build_cull leaves (same kind)
  if (!(recs_ready && mode == NDG_MODE_TC)) tr += launch_prep(N, pa, s);
  const int Ge = pa.Ge;
  int32_t* sv;
  long long* goff = (long long*)(w + L.goff);
  tr += backward_order(z, L, cull, Ge, w, !order_ready, s, &sv);
  BwdArgs ba{};
  ba.x = q->x;
  ba.dy = dy;
  ba.Q = q->Q;
  ba.tile = q->tile_size;
  ba.offsets = cull->offsets;
  ba.ids = cull->ids;
  ba.rec = pa.rec;
  ba.Ge = pa.Ge;
  ba.slot = nullptr;
  ba.part = (float*)(w + L.part);
  ba.status = pa.status;
  tr.begin();
  // tensor cores: the E Psi form for N <= 6, the beta form (bwd_hb.cu) above
  // (its operands fit shared and tensor memory up to N = 12)
  tr += mode == NDG_MODE_TC ? (N <= 6 ? launch_bwd_h(N, ba, z.T, s) : launch_bwd_hb(N, ba, z.T, s))
                            : launch_bwd(N, ba, z.T, s);
  tr.end();
  float* gsum = (float*)(w + L.gsum);
  tr += launch_segsum(ba.part, part_floats(N), goff, Ge, sv, cull->E_cap, pa.status, gsum, s);
  ChainArgs ch{};
  ch.G = mix->G;
  ch.has_children = mix->has_children;
  ch.gsum = gsum;
  ch.part_kind = mode == NDG_MODE_TC ? 1 : 0;
  ch.theta = mix->theta;
  ch.alpha_raw = mix->alpha_raw;
  ch.color_raw = mix->color_raw;
  ch.u_theta = mix->u_theta;
  ch.m_u = mix->m_u;
  ch.c_alpha_raw = mix->c_alpha_raw;
  ch.c_color_raw = mix->c_color_raw;
  ch.g_mean = grad->mean;
  ch.g_theta = grad->theta;
  ch.g_alpha = grad->alpha_raw;
  ch.g_color = grad->color_raw;
  ch.g_u_theta = grad->u_theta;
  ch.g_m_u = grad->m_u;
  ch.g_c_alpha = grad->c_alpha_raw;
  ch.g_c_color = grad->c_color_raw;
  tr += launch_chain(N, ch, s);
  return cuda_ok();
}

ndg_status ndg_adam(ndg_mixture* params, const ndg_mixture* grad, ndg_mixture* m1,
                    ndg_mixture* m2, int* step_dev, float lr, float beta1, float beta2, float eps,
                    ndg_stream stream, ndg_trace* trace) {
  ndg_status st;
  if ((st = check_mix(params)) || (st = check_mix(grad)) || (st = check_mix(m1)) ||
      (st = check_mix(m2)))
    return st;
  if (!step_dev) return NDG_ERR_INVALID_ARG;
  const ndg_mixture* all[4] = {params, grad, m1, m2};
  for (const ndg_mixture* m : all)
    if (m->N != params->N || m->G != params->G || m->has_children != params->has_children)
      return NDG_ERR_INVALID_ARG;
  const long long G = params->G, N = params->N, P = tri(params->N);
  AdamArgs a{};
  const long long width[8] = {N, P, 1, 3, P, N, 1, 3};
  float* pp[8] = {params->mean, params->theta, params->alpha_raw, params->color_raw,
                  params->u_theta, params->m_u, params->c_alpha_raw, params->c_color_raw};
  const float* gp[8] = {grad->mean, grad->theta, grad->alpha_raw, grad->color_raw,
                        grad->u_theta, grad->m_u, grad->c_alpha_raw, grad->c_color_raw};
  float* mp[8] = {m1->mean, m1->theta, m1->alpha_raw, m1->color_raw,
                  m1->u_theta, m1->m_u, m1->c_alpha_raw, m1->c_color_raw};
  float* vp[8] = {m2->mean, m2->theta, m2->alpha_raw, m2->color_raw,
                  m2->u_theta, m2->m_u, m2->c_alpha_raw, m2->c_color_raw};
  const int nseg = params->has_children ? 8 : 4;
  for (int i = 0; i < nseg; ++i) a.seg[i] = AdamSeg{pp[i], gp[i], mp[i], vp[i], G * width[i]};
  a.nseg = G > 0 ? nseg : 0;
  a.step = step_dev;
  a.lr = lr;
  a.b1 = beta1;
  a.b2 = beta2;
  a.eps = eps;
  Tracer tr(trace, (cudaStream_t)stream);
  tr.begin();
  tr += launch_adam(a, (cudaStream_t)stream);
  tr.end();
  return cuda_ok();
}

ndg_status ndg_densify(ndg_mixture* mix, float a_thr, float a_child0, const float* noise,
                       ndg_mixture* m1, ndg_mixture* m2, int* G_new_dev, void* ws,
                       size_t ws_bytes, ndg_stream stream, ndg_trace* trace) {
  ndg_status st;
  if ((st = check_mix(mix))) return st;
  if (!noise || !G_new_dev || !m1 || !m2) return NDG_ERR_INVALID_ARG;
  if (!mix->u_theta || !mix->m_u || !mix->c_alpha_raw || !mix->c_color_raw)
    return NDG_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, kAlign)) return NDG_ERR_INVALID_ARG;
  Sizes z = make_sizes(mix, nullptr, nullptr, 0);
  CommonLayout c = common_layout(z);
  if (ws_bytes < c.end) return NDG_ERR_WORKSPACE;
  char* w = (char*)ws;
  DensifyArgs a{};
  a.G = mix->G;
  a.G_cap = mix->G_cap;
  a.has_children = mix->has_children;
  a.a_thr = a_thr;
  a.a_child0 = a_child0;
  a.mean = mix->mean;
  a.theta = mix->theta;
  a.alpha_raw = mix->alpha_raw;
  a.color_raw = mix->color_raw;
  a.u_theta = mix->u_theta;
  a.m_u = mix->m_u;
  a.c_alpha_raw = mix->c_alpha_raw;
  a.c_color_raw = mix->c_color_raw;
  a.noise = noise;
  const ndg_mixture* moms[2] = {m1, m2};
  for (int i = 0; i < 2; ++i)
    a.mom[i] = MomentPtrs{moms[i]->mean, moms[i]->theta, moms[i]->alpha_raw, moms[i]->color_raw,
                          moms[i]->u_theta, moms[i]->m_u, moms[i]->c_alpha_raw,
                          moms[i]->c_color_raw};
  a.flag = (int*)(w + c.dflag);
  a.rank = (int*)(w + c.drank);
  a.fresh = (int*)(w + c.dfresh);
  a.G_new = G_new_dev;
  Tracer tr(trace, (cudaStream_t)stream);
  tr.begin();
  tr += launch_densify(mix->N, a, (cudaStream_t)stream);
  tr.end();
  return cuda_ok();
}

ndg_status ndg_probe_pipe(int which, int blocks, int threads, int iters, long long* cycles_dev,
                          float* sink_dev, ndg_stream stream) {
  if ((which != 0 && which != 1) || blocks < 1 || blocks > (1 << 20) || threads < 32 ||
      threads > 1024 || threads % 32 != 0 || iters < 1 || !cycles_dev || !sink_dev ||
      !aligned(cycles_dev, 8) || !aligned(sink_dev, 4))
    return NDG_ERR_INVALID_ARG;
  launch_probe_pipe(which, blocks, threads, iters, cycles_dev, sink_dev, (cudaStream_t)stream);
  return cuda_ok();
}

ndg_status ndg_read_status(void* ws, ndg_stream stream, int* device_status) {
  if (!ws || !device_status) return NDG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) return NDG_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, ws, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return NDG_ERR_CUDA;
  if (cudaMemset(ws, 0, sizeof(int)) != cudaSuccess) return NDG_ERR_CUDA;
  *device_status = v;
  return NDG_OK;
}

const char* ndg_status_string(int status) {
  switch (status) {
    case NDG_OK: return "ok";
    case NDG_ERR_INVALID_ARG: return "invalid argument";
    case NDG_ERR_CAPACITY: return "candidate capacity exceeded";
    case NDG_ERR_CUDA: return "CUDA error";
    case NDG_ERR_NUMERIC: return "non-finite parameter";
    case NDG_ERR_TIMEOUT: return "device wait timed out";
    case NDG_ERR_WORKSPACE: return "workspace too small";
    case NDG_ERR_SCRATCH_LIMIT: return "input exceeds the fixed no-allocation scratch";
    default: return "unknown status";
  }
}

int ndg_version(void) { return 1; }

}  // extern "C"
