// kernels.h -- argument blocks and launchers of the libndg kernels
// (internal; not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ndg {

struct PrepArgs {
  int G, Ge;
  const float *mean, *theta, *alpha_raw, *color_raw;
  const float *u_theta, *m_u, *c_alpha_raw, *c_color_raw;
  float* rec;  // [Ge][rec_floats(N)] or null
  int rec_kind;  // 0: M = L^-1 packed; 1: A = M^T M packed (lifted tensor-core form);
                 // 2: kind 1 followed by M (tensor-core backward; stride rec_tc_floats)
  // cull keys (when gkey or bin is set)
  int k, KP, B;
  const float* proj;
  float cutoff, k_sigma;
  float child_k_min;   // children's radius floor (Section 3.3), 0: none
  const float* range;  // lo, hi, inv_h, NDG_MAX_K each
  uint8_t* gkey;       // [Ge][2 KP] or null
  uint32_t* bin;       // [Ge] or null
  int* status;
  // Section 3.2 conditioning: when set, the inputs beyond position are the
  // constants xc [N - 3] and the keys are those of each Gaussian restricted
  // to them (position only); projections enter with their first 3 entries
  const float* xc;
};

struct CullTileArgs {
  const uint8_t* tkey;        // [T][2 KP]
  const uint8_t* gkey;        // [Ge][2 KP] in bin-sorted order (row p for sorted_ids[p])
  const long long* binoff;    // [nb * nb + 1]
  const int32_t* sorted_ids;  // Gaussians sorted by bin
  int B;
  long long* counts;          // count pass: [T][8] per warp slice
  const long long* excl;      // fill pass: exclusive scan of counts
  int* ids;                   // fill pass: [E_cap]
  long long E_cap;
  uint32_t* masks;            // [T][mask_words] survivor ballots of the count pass
  long long mask_words;       // per tile: >= ceil(max sources / 32) + 8
};

struct FwdArgs {
  const float* x;
  long long Q;
  int tile;
  const long long* offsets;  // [T+1]
  const int* ids;
  const float* rec;          // [Ge][rec_floats(N)]
  int Ge;
  float* y;                  // [Q][3]
  int* status;               // device status word (timeouts of bounded waits)
  int rec_stride4;           // float4s per record (0: the kernel's own record size)
  int mat_off4;              // FP32 form: float4 offset of M inside a record (0: M first)
  const int* tiles;          // null: CTA b is tile b; else CTA b < *n_tiles is tile tiles[b]
  const int* n_tiles;
};

// Many frames' tensor-core forwards in one persistent launch: the work list
// is every (frame, tile) item in frame order, taken with an atomic cursor.
struct FwdBatchArgs {
  const FwdArgs* frames;         // [n_frames] (tiles / n_tiles unused)
  const int* N;                  // [n_frames]
  const long long* tile_start;   // [n_frames + 1]: frame f owns items tile_start[f] ..
  unsigned long long* done;      // [n_frames] tiles completed (zero before the launch)
  unsigned long long* cursor;    // next item (zero before the launch)
  unsigned long long* stamps;    // [1 + n_frames] %globaltimer ns, or null: [0] first CTA
                                 // start (~0 before the launch), [1 + f] frame f complete
  int n_frames;
  long long n_items;
};

struct BwdArgs {
  const float* x;
  const float* dy;
  long long Q;
  int tile;
  const long long* offsets;
  const int* ids;
  const float* rec;
  int Ge;
  int* status;               // device status word (timeouts of bounded waits)
  const int32_t* slot;       // entry -> output record index, or null (entry order)
  float* part;               // [E_cap][part_floats(N)]
};

struct ChainArgs {
  int G, has_children;
  const float* gsum;         // [Ge][part_floats(N)]
  int part_kind;             // 0: [dl/dM, dl/dm, dl/dw]; 1: [G = dl/dA, v, dl/dw] with
                             //    dl/dM = 2 M G, dl/dm = 2 A v (A = M^T M)
  const float *theta, *alpha_raw, *color_raw, *u_theta, *m_u, *c_alpha_raw, *c_color_raw;
  float *g_mean, *g_theta, *g_alpha, *g_color, *g_u_theta, *g_m_u, *g_c_alpha, *g_c_color;
};

struct AdamSeg {
  float* p;
  const float* g;
  float* m;
  float* v;
  long long n;
};

struct AdamArgs {
  AdamSeg seg[8];
  int nseg;
  int* step;
  float lr, b1, b2, eps;
};

struct MomentPtrs {
  float *mean, *theta, *alpha_raw, *color_raw, *u_theta, *m_u, *c_alpha_raw, *c_color_raw;
};

struct DensifyArgs {
  int G, G_cap, has_children;
  float a_thr, a_child0;
  float *mean, *theta, *alpha_raw, *color_raw, *u_theta, *m_u, *c_alpha_raw, *c_color_raw;
  const float* noise;  // [G_cap][P + N + 4]
  MomentPtrs mom[2];
  int* flag;           // [G_cap] workspace
  int* rank;           // [G_cap] workspace
  int* fresh;          // [G_cap] workspace
  int* G_new;          // [1] caller
};

int launch_tile_bounds(int N, const float* x, long long Q, int tile, long long T, int k,
                        const float* proj, float* tb, cudaStream_t s, int nd = 0);  // nd: dims used (0: N)
int launch_cull_range(const float* tb, long long T, int k, int B, long long Q, float* range,
                       cudaStream_t s);
int launch_tile_keys(const float* tb, long long T, int k, int KP, int B, const float* range,
                      uint8_t* tkey, cudaStream_t s);
int launch_prep(int N, const PrepArgs& a, cudaStream_t s);
int launch_cull_tile(int KP, const CullTileArgs& a, long long T, cudaStream_t s);
int launch_permute_keys(const uint8_t* src, const int32_t* sorted, int n, int KP, uint8_t* dst,
                        cudaStream_t s);
int launch_tile_split(const long long* offsets, long long T, long long min_cand, int* la, int* lb,
                      int* n_a, int* n_b, cudaStream_t s);
int launch_fwd(int N, const FwdArgs& a, long long T, cudaStream_t s);
int launch_fwd_tc(int N, const FwdArgs& a, long long T, cudaStream_t s);  // FP16 hi/lo, N <= 12
unsigned fwd_tc_smem(int N);  // dynamic shared memory of the tensor-core forward for N (0: none)
int launch_fwd_tc_batch(const FwdBatchArgs& b, unsigned smem, int grid, cudaStream_t s);
int launch_bwd_h(int N, const BwdArgs& a, long long T, cudaStream_t s);   // N <= 6
int launch_bwd_hb(int N, const BwdArgs& a, long long T, cudaStream_t s);  // beta form, N <= 12
// n outputs; norm: the count the loss is normalised by (0: n)
int launch_loss(const float* y, const float* target, float* dy, long long n, double* part,
                double* loss, cudaStream_t s, double rel_eps = -1.0, long long norm = 0);
int launch_bwd(int N, const BwdArgs& a, long long T, cudaStream_t s);
int launch_selftest_wait(int* status, int which, cudaStream_t s);
int launch_segsum(const float* part, int RP, const long long* goff, int Ge, const int32_t* perm,
                  long long n_cap, int* status, float* gsum, cudaStream_t s);
int launch_chain(int N, const ChainArgs& a, cudaStream_t s);
int launch_adam(const AdamArgs& a, cudaStream_t s);
int launch_densify(int N, const DensifyArgs& a, cudaStream_t s);
int launch_probe_pipe(int which, int blocks, int threads, int iters, long long* cycles,
                      float* sink, cudaStream_t s);

}  // namespace ndg
