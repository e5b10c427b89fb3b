/*
 * ndg.h -- C ABI of libndg: evaluation, culling, back-propagation and
 * refinement of mixtures of N-dimensional Gaussians on one GB300 (sm_103a).
 *
 * Method: "N-Dimensional Gaussians for Fitting of High Dimensional
 * Functions" (SIGGRAPH 2024).  Each Gaussian has a mean m, a lower
 * triangular covariance factor L (V = L L^T, Section 3.1 Eq. 2) and an RGB
 * weight w = alpha c (Section 4.1 Eq. 8); the mixture value at a query x is
 *     y(x) = sum_g w_g exp(-1/2 (x - m_g)^T V_g^{-1} (x - m_g))   (Eq. 1, 8)
 * restricted, per tile of consecutive queries, to the Gaussians that survive
 * the random-projection cull of Section 3.2 (Eq. 3-5).
 *
 * Conventions shared by every entry point
 *   - Every pointer is caller-owned DEVICE memory unless stated otherwise;
 *     the library never allocates or frees memory and keeps no global
 *     state, with one documented exception: ndg_forward_noalloc's static
 *     scratch array.  Float arrays are FP32, row-major, contiguous, 4-byte
 *     aligned.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *     default stream).  Argument errors are detected on the host and
 *     returned before anything is launched.  Errors found on the device
 *     (capacity overflow, non-finite parameters) are written to a status
 *     word inside the workspace and read with ndg_read_status().
 *   - `ws` is scratch device memory of at least ndg_workspace_size() bytes
 *     (256-byte aligned).  Calls that share a workspace must be ordered (one
 *     stream, or events between streams), with one exception:
 *     ndg_backward_order writes only the backward's part of the workspace
 *     and may run concurrently with ndg_forward and the loss calls (not with
 *     ndg_build_cull, ndg_backward or ndg_densify).
 *   - Raw parameters (per parent row g, G rows in use, G_cap allocated):
 *       mean      [G_cap][N]
 *       theta     [G_cap][P]  P = N(N+1)/2, packed lower triangle row by
 *                             row: entry (i,j), j <= i, at i(i+1)/2 + j.
 *                             L_ii = exp(theta), L_ij = 2 sigmoid(theta) - 1
 *                             (Section 3.1; the paper's "i<j" read as the
 *                             strictly lower entries)
 *       alpha_raw [G_cap]     brightness alpha = exp(a)      (Section 4.1)
 *       color_raw [G_cap][3]  colour c = sigmoid(gamma)      (Section 4.1)
 *     and, when has_children != 0, one child per parent (Section 3.3,
 *     Eq. 6-7: L_c = L_p U, m_c = L_p m_u + m_p), same shapes:
 *       u_theta [G_cap][P], m_u [G_cap][N], c_alpha_raw [G_cap],
 *       c_color_raw [G_cap][3].
 *     Evaluated Gaussians: Ge = G (1 + has_children); index e < G is parent
 *     e, index e >= G is the child of parent e - G.
 *   - Queries: Q points x [Q][N]; tile t holds queries
 *     [t tile_size, min(Q, (t+1) tile_size)), T = ceil(Q / tile_size).
 *     Tiles are the unit of culling (Section 3.2: 16 x 16 pixel tiles), so
 *     consecutive queries should be close (image tiles, Morton order).
 */
#ifndef NDG_H
#define NDG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NDG_OK = 0,
  NDG_ERR_INVALID_ARG = 1, /* bad size, NULL or misaligned pointer       */
  NDG_ERR_CAPACITY = 2,    /* candidate entries exceeded E_cap           */
  NDG_ERR_CUDA = 3,        /* a CUDA launch or copy failed               */
  NDG_ERR_NUMERIC = 4,     /* non-finite activated value (L, m or w) of an
                              evaluated Gaussian                          */
  NDG_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out         */
  NDG_ERR_WORKSPACE = 6,   /* ws smaller than ndg_workspace_size()       */
  NDG_ERR_SCRATCH_LIMIT = 7 /* input larger than ndg_forward_noalloc's
                               fixed scratch (NDG_NOALLOC_SCRATCH_BYTES)  */
} ndg_status;

#define NDG_MAX_N 12      /* dimensions                                  */
#define NDG_MAX_K 32      /* random projections                          */
#define NDG_MAX_BUCKETS 255
#define NDG_MAX_TILE 256  /* queries per tile                            */

typedef void* ndg_stream; /* a cudaStream_t */

/* Raw mixture parameters (layouts above).  The same struct describes
 * gradients and Adam moments, which share the parameters' layout. */
typedef struct {
  int N, G, G_cap, has_children;
  float *mean, *theta, *alpha_raw, *color_raw;
  float *u_theta, *m_u, *c_alpha_raw, *c_color_raw;
} ndg_mixture;

typedef struct {
  long long Q;      /* number of queries (>= 0)                           */
  int tile_size;    /* 1 .. NDG_MAX_TILE                                  */
  const float* x;   /* [Q][N] device                                      */
} ndg_queries;

/* Section 3.2: k random unit vectors r_j (rows of proj, [k][N] device).  A
 * Gaussian is dropped for a tile when, for some j, the tile's projected
 * queries lie outside m_r +- k_g sigma_r (Eq. 3-5, "outside" per the text
 * around Eq. 5).  k_g = k_sigma (the paper uses 3) when cutoff == 0;
 * with cutoff > 0, k_g = sqrt(2 ln(max_c w_gc / cutoff)) so that every
 * dropped contribution is below cutoff, and a Gaussian whose largest weight
 * is below cutoff is dropped everywhere.  k == 0 keeps every live Gaussian
 * in every tile (dense evaluation).  The decision follows an integer bucket
 * contract over `buckets` (1 .. NDG_MAX_BUCKETS) buckets per projection
 * that is reproducible bit for bit and never drops a pair the real-valued
 * test keeps. */
typedef struct {
  int k;
  const float* proj;
  float cutoff;
  float k_sigma;
  int buckets;
  /* Section 3.3: a child (evaluated index >= G) starts with a negligible
   * contribution spanning its parent and is optimised until it
   * materialises; with child_k_min > 0 its radius is at least child_k_min
   * (e.g. the 3 of Eq. 5) even when its largest weight is below the cutoff,
   * so that it is evaluated, and receives a gradient, where it spans the
   * parent (a wider radius only keeps more pairs: every dropped contribution
   * stays below the cutoff).  0: no floor. */
  float child_k_min;
} ndg_cull_params;

/* Candidate lists as CSR over tiles.  Caller-owned device buffers:
 * offsets [T+1] (int64), ids [E_cap] (int32 evaluated-Gaussian indices),
 * E_dev [1] (int64, the true total, which may exceed E_cap).  Offsets are
 * clamped to E_cap, so a truncated list never indexes past the buffer. */
typedef struct {
  long long* offsets;
  int* ids;
  long long E_cap;
  long long* E_dev;
} ndg_cull;

/* Optional per-call trace (every entry point that launches work takes one;
 * NULL disables it).  main_begin / main_end are cudaEvent_t handles (or
 * NULL) recorded on the call's stream immediately before and after its main
 * kernel: the per-tile cull (fill pass) of ndg_build_cull, the evaluation
 * of ndg_forward, the per-pair partials of ndg_backward, the update of
 * ndg_adam, the selection of ndg_densify, the reduction of ndg_loss_l2.
 * `launches` is increased by the number of kernels the call launched. */
typedef struct {
  void* main_begin;
  void* main_end;
  long long launches;
} ndg_trace;

/* Bytes of workspace needed by every call below for these sizes.
 * E_cap bounds the candidate entries ndg_backward may see. */
size_t ndg_workspace_size(const ndg_mixture* mix, const ndg_queries* q,
                          const ndg_cull_params* cp, long long E_cap);

/* Section 3.2 (Eq. 3-5): build the per-tile candidate lists.  Order inside
 * a tile is deterministic (by first-projection bucket range, then index).
 * Device errors: NDG_ERR_CAPACITY when more than E_cap entries exist (the
 * lists are truncated, *E_dev holds the true total). */
ndg_status ndg_build_cull(const ndg_mixture* mix, const ndg_queries* q,
                          const ndg_cull_params* cp, ndg_cull* out, void* ws,
                          size_t ws_bytes, ndg_stream stream, ndg_trace* trace);

/* Section 3.2, the case of inputs beyond position constant for an image:
 * the same lists as ndg_build_cull, but each Gaussian is first restricted to
 * the constant inputs xc = (x_4 .. x_N) [N - 3] (device pointer): with the
 * precision A = (L L^T)^-1 split into position (first three inputs) and the
 * rest, completing the square turns it into a 3-D Gaussian over position
 * with weight w exp(-q_c / 2) (q_c = d_c^T A_cc d_c - b^T A_pp^-1 b,
 * b = A_pc d_c, d_c = xc - m_c), mean m_p - A_pp^-1 b and covariance A_pp^-1.
 * Keys, cutoff radius and tile bounds then use position only: the first
 * three entries of each projection and of each query (the caller's queries
 * must carry xc in their other inputs; they are not read).  The lists are
 * exactly those of the contract on the restricted Gaussians and are usually
 * far shorter than on all N inputs.  N >= 4, else NDG_ERR_INVALID_ARG;
 * evaluation (ndg_forward / ndg_backward) is unchanged. */
ndg_status ndg_build_cull_conditioned(const ndg_mixture* mix, const ndg_queries* q,
                                      const ndg_cull_params* cp, const float* xc,
                                      ndg_cull* out, void* ws, size_t ws_bytes,
                                      ndg_stream stream, ndg_trace* trace);

#define NDG_MODE_FP32 0 /* centred form z = L^{-1}(x - m) on the FP32 pipe */
#define NDG_MODE_TC 1   /* lifted quadratic form on the tensor cores: s =
                           phi(x - c) . coef with phi = [x x^T (lower), x, 1]
                           about the tile centre c, coef from A = V^-1; FP16
                           hi/lo operands (3 products) with exact power-of-two
                           scaling, FP32 accumulation; N <= 12; outputs within
                           ~2e-4 relative of the FP64 definition */
#define NDG_MODE_AUTO 2 /* forward: per tile, NDG_MODE_TC where the tile has
                           at least NDG_AUTO_MIN_CANDIDATES(N) candidates (the
                           contraction is dense enough for 128-candidate
                           tensor-core chunks), NDG_MODE_FP32 elsewhere; each
                           tile's outputs equal those of the mode it gets.
                           backward: NDG_MODE_TC */
/* Crossover measured on GB300 with full tiles of 256 queries: the two forms
 * take equal time at about 190 candidates per tile for N = 6 and about 110
 * for N = 10. */
#define NDG_AUTO_MIN_CANDIDATES(N) ((N) <= 6 ? 192 : 128)

/* Mode flag for ndg_forward and ndg_backward (and ndg_frame.flags): the
 * prepared per-Gaussian records in `ws` are those that ndg_build_cull (or
 * ndg_build_cull_conditioned) wrote there from these same parameters, and
 * no call on this workspace since has prepared records itself (an
 * ndg_forward or ndg_backward without this flag rewrites them in its own
 * layout); the call then skips its own preparation (the values are the same
 * either way).  ndg_backward uses it in NDG_MODE_TC and ignores it in
 * NDG_MODE_FP32. */
#define NDG_RECORDS_READY 0x200

/* Eq. 1 and Eq. 8: y [Q][3] = culled mixture sum at every query.  `cull`
 * must come from ndg_build_cull on the same mixture and queries.  mode:
 * NDG_MODE_FP32, NDG_MODE_TC or NDG_MODE_AUTO (else NDG_ERR_INVALID_ARG),
 * optionally with NDG_RECORDS_READY. */
ndg_status ndg_forward(const ndg_mixture* mix, const ndg_queries* q,
                       const ndg_cull* cull, int mode, float* y, void* ws,
                       size_t ws_bytes, ndg_stream stream, ndg_trace* trace);

/* Plain L2 loss over the Q x 3 outputs (the paper trains with a relative L2,
 * Section 4.1; the plain form is the one used here):
 *   loss = sum (y - target)^2 / (3Q) written to loss_dev [1] (FP64),
 *   dy = 2 (y - target) / (3Q)  [Q][3].  Deterministic reduction. */
ndg_status ndg_loss_l2(long long Q, const float* y, const float* target,
                       float* dy, double* loss_dev, void* ws, size_t ws_bytes,
                       ndg_stream stream, ndg_trace* trace);

/* The plain L2 loss of one shard of a larger query set, for a fit whose
 * queries are split across processes (one per GPU): the Q outputs given
 * here are normalised by the whole set's Q_total (>= Q), so that
 *   loss_dev [1] = sum (y - target)^2 / (3 Q_total)   (this shard's share),
 *   dy = 2 (y - target) / (3 Q_total)  [Q][3];
 * the shards' losses and gradients then add up to those of the whole set.
 * Q_total == Q is ndg_loss_l2.  The paper has no multi-GPU fit; this is the
 * query-sharded data parallelism of this library (tiles are independent in
 * the cull and the evaluation, Section 3.2 and Eq. 8). */
ndg_status ndg_loss_l2_shard(long long Q, long long Q_total, const float* y, const float* target,
                             float* dy, double* loss_dev, void* ws, size_t ws_bytes,
                             ndg_stream stream, ndg_trace* trace);

/* Relative L2 loss.  Section 4.1 trains with a relative L2 loss (after
 * Noise2Noise) without printing its form; the reading implemented:
 *   loss = sum (y - target)^2 / (y^2 + eps) / (3Q) written to loss_dev [1]
 *   (FP64), dy = 2 (y - target) / (y^2 + eps) / (3Q)  [Q][3],
 * the denominator treated as a constant when differentiating (no gradient
 * flows through it).  eps > 0 (finite), e.g. 1e-2; otherwise
 * NDG_ERR_INVALID_ARG.  Deterministic reduction; same workspace use as
 * ndg_loss_l2. */
ndg_status ndg_loss_rel_l2(long long Q, const float* y, const float* target,
                           float eps, float* dy, double* loss_dev, void* ws,
                           size_t ws_bytes, ndg_stream stream, ndg_trace* trace);

/* The Gaussian-major order of `cull`'s entries that ndg_backward sums the
 * per-entry gradient records in (a stable transposition of the candidate
 * lists: per Gaussian, its entries in tile order), written into the
 * backward's part of `ws` (same size rule as ndg_backward).  It depends on
 * the lists only, so it can run on another stream while the forward and the
 * loss run; ndg_backward with mode | NDG_BWD_ORDER_READY then uses it
 * instead of recomputing it.  The caller orders the two calls (an event)
 * and passes the same mix sizes, q, cull and ws to both.  Same argument
 * errors as ndg_backward's. */
ndg_status ndg_backward_order(const ndg_mixture* mix, const ndg_queries* q, const ndg_cull* cull,
                              void* ws, size_t ws_bytes, ndg_stream stream, ndg_trace* trace);

/* Flag for ndg_backward's mode: the order of ndg_backward_order is already
 * in ws for this cull.  An order left from other lists cannot make the
 * backward read outside the workspace (indices are bounds-checked, and an
 * index out of range sets NDG_ERR_INVALID_ARG in the status word), but its
 * gradients are then wrong. */
#define NDG_BWD_ORDER_READY 0x100

/* Analytic gradient of the loss through Eq. 1, 2, 6-8 given dy = dl/dy
 * [Q][3]: writes dl/d(raw parameter) into `grad` (same layout and N, G,
 * has_children as mix; rows >= G untouched).  Recomputes everything from
 * the raw parameters and `cull`; per-Gaussian sums run in a fixed order
 * (no atomics), so results are bit-reproducible.  Requires E < 2^31.
 * mode NDG_MODE_FP32: centred form on the FP32 pipe; NDG_MODE_TC: the
 * lifted form on the tensor cores, every N (for N <= 6 the gradients of the
 * lifted coefficients and of w come from a second contraction E Psi with
 * Psi = dy (x) phi; above, from beta Phi with beta = e sum_c dy_c w_c and
 * dl/dw summed in FP32); NDG_MODE_AUTO: NDG_MODE_TC; any of them may carry
 * NDG_BWD_ORDER_READY and NDG_RECORDS_READY.  Tensor-core gradients are within ~6e-4 relative of
 * the FP64 definition per tensor. */
ndg_status ndg_backward(const ndg_mixture* mix, const ndg_queries* q,
                        const ndg_cull* cull, int mode, const float* dy,
                        ndg_mixture* grad, void* ws, size_t ws_bytes,
                        ndg_stream stream, ndg_trace* trace);

/* Adam (Kingma & Ba) over every raw parameter of rows < G (children too
 * when has_children); the paper does not name its optimiser.  m1, m2 are
 * the first and second moments in the parameters' layout; step_dev [1] is
 * the device step counter t (read as t, the update uses t + 1, then it is
 * incremented), so the call can be captured in a CUDA graph. */
ndg_status ndg_adam(ndg_mixture* params, const ndg_mixture* grad,
                    ndg_mixture* m1, ndg_mixture* m2, int* step_dev, float lr,
                    float beta1, float beta2, float eps, ndg_stream stream,
                    ndg_trace* trace);

/* Section 3.3 refinement.  Children whose raw brightness exceeds
 * a_thr = (float) ln t materialise as new parents appended at rows
 * G .. G_new-1 (L = L_p U written back to raw form with off-diagonals
 * clamped to +-(1 - 1e-6), m = L_p m_u + m_p, the child's own brightness
 * and colour); at most G_cap - G do, the brightest first, ties at the
 * boundary all left out.  Every materialised parent and new row receives a
 * fresh child from its row of `noise` [G_cap][P + N + 4] (standard
 * normals): u_theta = 0.05 xi, m_u = 0.1 xi, c_alpha_raw = a_child0 +
 * 0.1 xi, c_color_raw = own colour + 0.1 xi; Adam moments of every touched
 * row are zeroed.  With has_children == 0 every parent receives a child and
 * nothing materialises.  G_new_dev [1] receives the new row count; the
 * caller sets mix->G and has_children = 1 for later calls. */
ndg_status ndg_densify(ndg_mixture* mix, float a_thr, float a_child0,
                       const float* noise, ndg_mixture* m1, ndg_mixture* m2,
                       int* G_new_dev, void* ws, size_t ws_bytes,
                       ndg_stream stream, ndg_trace* trace);

/* ndg_forward without a workspace, for callers that cannot allocate device
 * memory (for example a plugin inside a host application whose allocator
 * owns the whole device budget, or a per-frame callback that cannot afford
 * the device synchronisation an allocation may cause).  The paper has no
 * counterpart; it is a deployment convenience.  Same result as ndg_forward
 * (mode NDG_MODE_FP32) on the same inputs; the caller still owns mix, q,
 * cull and y.  Argument errors (sizes, NULL or misaligned pointers) are the
 * same as ndg_forward's and return NDG_ERR_INVALID_ARG before anything runs;
 * cull->E_dev is not read.  Its scratch (the prepared records, Ge * R * 4
 * bytes with Ge = G (1 + has_children) and R = N(N+1)/2 + N + 3 rounded up
 * to a multiple of 4) lives in one static device array of
 * NDG_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * exit; larger mixtures return NDG_ERR_SCRATCH_LIMIT before anything runs
 * (N = 6: up to 131072 evaluated Gaussians; N = 10: up to 61680).  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process, so make
 * that first call before any stream capture, and do not call this entry
 * point on a device after cudaDeviceReset.  All calls share the array:
 * calls that overlap on the GPU race and must be serialised by the caller.
 * NDG_ERR_CUDA reports a launch failure of this call only (an error left
 * pending by an earlier call is neither reported nor cleared).  Device-side
 * status (non-finite parameters) is not reported by this variant.  Calls
 * nothing that allocates. */
#define NDG_NOALLOC_SCRATCH_BYTES (16 << 20)
ndg_status ndg_forward_noalloc(const ndg_mixture* mix, const ndg_queries* q,
                               const ndg_cull* cull, float* y, ndg_stream stream);

/* One frame of a batched render: ndg_forward's arguments for that frame. */
typedef struct ndg_frame {
  const ndg_mixture* mix;
  const ndg_queries* q;
  const ndg_cull* cull; /* from ndg_build_cull on this mix and q */
  float* y;             /* [Q][3] */
  void* ws;             /* this frame's workspace: at least
                           ndg_workspace_size(mix, q, NULL, 0) bytes */
  size_t ws_bytes;
  int flags;            /* 0, or NDG_RECORDS_READY: the records this
                           frame's cull left in ws are current */
} ndg_frame;

/* Bytes of the batch descriptor workspace of ndg_forward_batch. */
size_t ndg_batch_workspace_size(int n_frames);

/* Eq. 1 and Eq. 8 for many frames (mixtures and query sets of uneven size,
 * 1 <= N <= 12 each) in one persistent launch of the tensor-core form.  The
 * work list is every (frame, query tile) in the order of `frames`; one CTA
 * per SM takes the next item with an atomic cursor, so a frame's last tiles
 * overlap the next frame's first ones.  Each frame's y equals that of
 * ndg_forward(..., NDG_MODE_TC, ...) on the same frame, bit for bit.
 *   frames    HOST array [n_frames] (read during the call only); frames with
 *             Q = 0 contribute no work.
 *   batch_ws  device, >= ndg_batch_workspace_size(n_frames) bytes, 256-byte
 *             aligned; holds the work list (written by a host-to-device
 *             copy issued on `stream`).
 *   stamps    device [1 + n_frames] or NULL: %globaltimer nanoseconds;
 *             stamps[0] the start of the first CTA, stamps[1 + f] the moment
 *             the last tile of frame f completed (0 for an empty frame).
 * Each frame's status (non-finite parameters, timed-out waits) goes to its
 * own workspace (ndg_read_status on frames[f].ws).  Argument errors of any
 * frame return NDG_ERR_INVALID_ARG (NDG_ERR_WORKSPACE for a short ws)
 * before anything runs. */
ndg_status ndg_forward_batch(const ndg_frame* frames, int n_frames, void* batch_ws,
                             size_t batch_ws_bytes, unsigned long long* stamps,
                             ndg_stream stream, ndg_trace* trace);

/* Failure-detection self-test of the bounded device waits: launches one
 * CTA that waits on an mbarrier nothing ever completes, with the wait the
 * tensor-core kernels use (which = 0: the sleeping warp wait, about a
 * second; which = 1: the spinning wait of their final drain, about a second
 * or two).  When the bound runs out it records NDG_ERR_TIMEOUT in the
 * workspace status word (read with ndg_read_status) and returns; nothing
 * faults and the context stays usable.  ws: any workspace (only its status
 * word is used). */
ndg_status ndg_selftest_timeout(int which, void* ws, size_t ws_bytes, ndg_stream stream);

/* Measurement helper (no counterpart in the paper): throughput probe of one
 * arithmetic pipe, for the rooflines the benchmark reports.  which = 0: the
 * MUFU exponential (ex2.approx, one per Gaussian-query pair in every
 * evaluation kernel); which = 1: the FP32 FMA.  Launches `blocks` blocks of
 * `threads` threads (a multiple of 32, at most 1024), at most one block per
 * SM at a time; every thread executes 8 x iters dependent instructions in 8
 * independent chains.  cycles_dev [blocks] receives each block's clock64
 * cycles around its loop, sink_dev [blocks * threads] the chains' results
 * (so nothing is optimised away).  Rate per SM per clock = threads * 8 *
 * iters / cycles. */
ndg_status ndg_probe_pipe(int which, int blocks, int threads, int iters, long long* cycles_dev,
                          float* sink_dev, ndg_stream stream);

/* Synchronises `stream`, copies the workspace status word to *device_status
 * (an ndg_status value) and clears it. */
ndg_status ndg_read_status(void* ws, ndg_stream stream, int* device_status);

const char* ndg_status_string(int status);
int ndg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NDG_H */
