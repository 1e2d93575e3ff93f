/*
 * gft.h -- C ABI of the GB300 batched fast graph Fourier transform.
 *
 * Method: Lu & Ortega, "Fast Graph Fourier Transforms Based on Graph
 * Symmetry and Bipartition".  The GFT of a signal x on a graph with
 * Laplacian L = U diag(lambda) U^T is U^T x (Sec. II-B).  When the graph is
 * symmetric under a node involution phi (Definition 2), one stage of Haar
 * units B_phi (Eq. 20) block-diagonalises L into the Laplacians of two
 * smaller graphs G+ and G- (Thm. 3, Eq. 17), so U = B_phi diag(U+, U-)
 * (Eq. 13); repeating on G+ and G- gives several stages (end of Sec. IV-C).
 * A plan holds the stages and the dense bases U_k of the leaf blocks; the
 * forward transform applies the stages (additions and subtractions only,
 * the 1/sqrt(2) factors folded into the U_k, Sec. III) and then the block
 * products U_k^T, and writes the coefficients in ascending eigenvalue order.
 * Bipartite graphs give the mirror image, a stage of Haar units on the
 * OUTPUT side after two sub-transforms (Sec. III-A, gft_plan_create_bipartite);
 * gft_approx_* replaces the leaves' dense products by greedy layers of
 * Givens rotations (the comparison of Sec. VI-B), and gft_givens_* applies
 * and trains layered Givens surrogates.
 *
 * Conventions shared by every call:
 *  - Signals are rows: a batch is a row-major [batch, n] array, one signal
 *    per row; coefficients likewise (y = x U per row, i.e. y^T = U^T x).
 *  - Node labels are 0-based.
 *  - Device pointers must be 16-byte aligned and point to memory of the
 *    current CUDA device; in-place (x == y) is allowed for plan transforms.
 *  - Streams are passed as an opaque pointer holding a cudaStream_t
 *    (NULL = the legacy default stream).  Transform calls are asynchronous
 *    with respect to the host; errors raised by a kernel surface through
 *    gft_device_error() or the next synchronising call.
 *  - Every call returns a gft_status and never aborts or throws across the
 *    ABI.  A call that fails validation writes nothing to its outputs.
 *  - Objects are not thread-safe: do not use one plan from two host threads
 *    at the same time.
 */
#ifndef GFT_H
#define GFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gft_plan_s* gft_plan_t;
typedef struct gft_batch_s* gft_batch_t;
typedef struct gft_givens_s* gft_givens_t;
typedef struct gft_approx_s* gft_approx_t;
typedef void* gft_stream_t;

typedef enum {
    GFT_OK = 0,
    GFT_ERR_INVALID_ARG = 1,     /* null pointer, bad size, bad flag, bad stage count */
    GFT_ERR_NOT_INVOLUTION = 2,  /* phi(phi(i)) != i or label out of range (Definition 1) */
    GFT_ERR_NOT_SYMMETRIC = 3,   /* block Laplacian not phi-symmetric (Definition 2) */
    GFT_ERR_NOT_LAPLACIAN = 4,   /* L not symmetric or has a non-finite entry */
    GFT_ERR_NO_CONVERGENCE = 5,  /* Jacobi exceeded its sweep limit */
    GFT_ERR_CUDA = 6,            /* a CUDA runtime call failed */
    GFT_ERR_OOM = 7,             /* device or host allocation failed */
    GFT_ERR_TIMEOUT = 8,         /* a bounded device-side wait gave up */
    GFT_ERR_UNSUPPORTED = 9,     /* valid input the library does not handle (see message) */
    GFT_ERR_MISALIGNED = 10,     /* device pointer not 16-byte aligned */
    GFT_ERR_BLOCK_LEAK = 11,     /* a stage involution maps a node out of its block */
    GFT_ERR_NO_DEVICE = 12,      /* plan was created with GFT_ANALYZE_ONLY */
    GFT_ERR_NOT_BIPARTITE = 13   /* no right Haar stage: odd cycle, or part blocks not alpha*I */
} gft_status;

/* gft_plan_create flags */
#define GFT_SPLIT_COMPONENTS 0x1u  /* split leaves into connected components (Sec. V-E) */
#define GFT_ORDER_BLOCK      0x2u  /* coefficients in leaf order instead of ascending eigenvalue */
#define GFT_ANALYZE_ONLY     0x4u  /* host-side decomposition only: no device, no bases */
#define GFT_NO_JIT           0x8u  /* never build plan-specialised kernels (interpreter only) */
#define GFT_KERNEL_TABLE     0x10u /* CUDA-core transforms: the table-driven kernel wherever
                                      it fits (leaves of at most 64 nodes) */
#define GFT_KERNEL_WIDE      0x20u /* CUDA-core transforms: the wide-leaf kernel whenever the
                                      plan has a leaf of more than 32 nodes */
#define GFT_SEARCH_STAGES    0x40u /* n_stages = 0: find the stages with gft_search_stages
                                      (up to 16 stages, 10^6 search steps each).  When the
                                      step budget runs out, the search keeps the stages
                                      found so far (possibly none) and the plan is still
                                      created: read the stage count back from
                                      gft_plan_get_info (info.n_stages). */
#define GFT_NORMALIZED       0x80u /* transform with the normalised Laplacian D^-1/2 L D^-1/2
                                      (d_i = l_ii > 0) of the given L (Sec. II-B) */

/* transform precision (plan forward / inverse) */
#define GFT_PREC_FP32    0u  /* CUDA-core FP32 FMA, FP32 accumulation */
#define GFT_PREC_BF16    1u  /* leaf products on tensor cores, BF16 operands */
#define GFT_PREC_BF16X3  2u  /* BF16 hi+lo split, three products (hi*hi + hi*lo + lo*hi) */
#define GFT_PREC_FP16X3  3u  /* FP16 hi+lo split (scaled), three products */
#define GFT_BATCH_NO_JIT 0x100u /* mixed batches: no plan-specialised group (or'ed into the precision) */

/* Human-readable name of a status code (static string, never NULL). */
const char* gft_status_string(gft_status s);

/* Text of the last error raised on this host thread (static storage,
 * overwritten by the next failing call; "" if none). */
const char* gft_last_error(void);

/* ABI version: major*10000 + minor*100 + patch. */
int32_t gft_version(void);

/*
 * Laplacian from weights, Eq. 5 (Sec. II-B): l_ii = s_i + sum_{j != i} w_ij,
 * l_ij = -w_ij.  W: host, n*n row-major, symmetric, diagonal ignored;
 * s: host, n self-loop weights (NULL = none); L: host, n*n output.  The
 * caller owns all three.  Errors: INVALID_ARG on null W/L or n < 1,
 * NOT_LAPLACIAN if W is not symmetric or not finite.
 */
gft_status gft_laplacian_from_weights(int32_t n, const double* W, const double* s, double* L);

/*
 * Symmetric normalised Laplacian D^-1/2 L D^-1/2 (Sec. II-B) of the graph
 * (W, s) as in gft_laplacian_from_weights, d_i = l_ii.  Errors as there,
 * plus NOT_LAPLACIAN for a node without positive degree.
 */
gft_status gft_normalized_laplacian_from_weights(int32_t n, const double* W, const double* s, double* L);

/*
 * Build a fast-GFT plan (Sec. IV-B, IV-C; recursion at the end of Sec. IV-C).
 *  n         number of nodes, 1 <= n <= 4096.
 *  L         host, n*n row-major Laplacian (Eq. 3), copied.  Must be
 *            symmetric and finite; signs of entries are not checked, so
 *            negative weights (as in G+/G-) are accepted.
 *  n_stages  number of Haar stages, 0 <= n_stages <= 16 (0 = dense GFT).
 *  phi       host, n_stages*n involutions on ORIGINAL labels, copied
 *            (NULL allowed when n_stages = 0).  Stage s splits every current
 *            block that phi_s moves: phi_s must map each block onto itself,
 *            the block's Laplacian must satisfy l_ij = l_phi(i)phi(j) within
 *            1e-12*max(1,max|L|), and paired nodes must have taken part in
 *            the same number of earlier stages (else UNSUPPORTED).  In each
 *            block, the pair member that comes first in the block's order
 *            goes to X, its partner to Y; G+ lists X then the fixed points Z,
 *            G- lists the partners of X in X's order.
 *  flags     GFT_SPLIT_COMPONENTS | GFT_ORDER_BLOCK | GFT_ANALYZE_ONLY | GFT_NO_JIT |
 *            GFT_KERNEL_TABLE | GFT_KERNEL_WIDE (these two are exclusive) |
 *            GFT_SEARCH_STAGES (with n_stages = 0 and phi = NULL: the stages
 *            gft_search_stages finds, Sec. V-F) | GFT_NORMALIZED (the plan is
 *            built for D^-1/2 L D^-1/2, d_i = l_ii, which must be positive;
 *            NOT_LAPLACIAN otherwise).  Stage involutions must then be
 *            symmetries of the normalised matrix, which holds for every
 *            symmetry of the graph since degrees are invariant.
 *  out       receives the plan (owned by the caller; free with
 *            gft_plan_destroy).  Unchanged on error.
 * Unless GFT_ANALYZE_ONLY is set, the leaf Laplacians are eigendecomposed on
 * the current CUDA device by a batched FP64 Jacobi kernel and the bases are
 * uploaded; the call synchronises the device.  For graphs of at most 128
 * nodes (sum of squared leaf sizes <= 8192; <= 4096 for the FP64 kernel)
 * and without GFT_NO_JIT, the call also generates a kernel specialised to
 * this plan (indices and folded leaf matrices as constants), compiles it
 * with NVRTC for sm_103a, and times several launch shapes on a scratch
 * batch to keep the fastest; transforms then use it.  The tensor-core data (pre-split leaf bases) is
 * built on the first tensor-core transform; make that first call outside
 * any stream capture.  Otherwise, when some leaf has more than 32 nodes
 * (up to 512), a wide-leaf kernel computes each tile's leaf products as a
 * register-blocked GEMM of the whole CTA; for leaves of at most 64 nodes the
 * call times it against the table-driven kernel and keeps the faster
 * (GFT_KERNEL_TABLE / GFT_KERNEL_WIDE force one).  Eigenvector signs: the first
 * significant entry (magnitude above 1e-8 of the vector's largest) of every
 * full-length basis vector is made positive, which keeps the closed forms'
 * own signs (DCT-II of a uniform path, the printed 4-cycle basis).  Output order: ascending eigenvalue;
 * eigenvalues within 1e-9*max(1,|lambda|max) of a neighbour form a cluster
 * ordered by (leaf in depth-first order with + before -, index in leaf).
 * Errors: INVALID_ARG, NOT_LAPLACIAN, NOT_INVOLUTION, BLOCK_LEAK,
 * NOT_SYMMETRIC, UNSUPPORTED, NO_CONVERGENCE, CUDA, OOM.
 */
gft_status gft_plan_create(int32_t n, const double* L, int32_t n_stages, const int32_t* phi,
                           uint32_t flags, gft_plan_t* out);

/*
 * Build `count` plans at once (same meaning per plan as gft_plan_create):
 * n[i], L[i] (host pointers), n_stages[i], phi[i] (host pointer, NULL when
 * n_stages[i] = 0; phi itself may be NULL when every n_stages[i] = 0).  The
 * graphs are decomposed on the host and the leaves of ALL of them are
 * eigendecomposed in one batched FP64 Jacobi solve on the device (leaves
 * grouped by size; the largest on their own stream), which is what makes
 * building thousands of plans practical.  All or nothing: on any error no
 * plan is returned and out is unchanged.  out[count] receives the plans.
 */
gft_status gft_plan_create_many(int32_t count, const int32_t* n, const double* const* L,
                                const int32_t* n_stages, const int32_t* const* phi, uint32_t flags,
                                gft_plan_t* out);

/*
 * Bipartite plan with a right Haar stage (Sec. III-A, Lemma 1, Thms. 1-2):
 * U^T x = B_{n,p} diag(E^T, F^T) x (Eq. 8).  L must split into two parts
 * S1, S2 with L[S1,S1] = L[S2,S2] = alpha*I (within 1e-12*max(1,max|L|)):
 * the Laplacian of a k-regular bipartite graph (alpha = k) or the
 * normalised Laplacian of any bipartite graph (alpha = 1).  With the
 * coupling block C = -L[S1,S2], E holds the left singular vectors of C on
 * the larger part, F the right singular vectors on the smaller part
 * (p = its size); unit c pairs column c of E and of F: coefficient
 * (e_c.x + f_c.x)/sqrt2 has eigenvalue alpha - sigma_c, (e_c.x - f_c.x)/sqrt2
 * has alpha + sigma_c; E's columns beyond p have eigenvalue alpha.  The
 * singular vectors come from the FP64 Jacobi eigendecomposition of
 * [[0, C], [C^T, 0]] on the device (no squaring of C); singular values below
 * 1e-9*max(1, sigma_max) count as zero and their vectors are separated by
 * pivoted Gram-Schmidt.
 *  n, L      as gft_plan_create.
 *  side      NULL (parts found by two-colouring the nonzero off-diagonal
 *            pattern; colour 0 for each component's smallest node), or n
 *            entries 0 / 1.  The larger part is E's (colour 0 on a tie);
 *            within a part, nodes are in ascending label order.
 *  flags     GFT_ORDER_BLOCK | GFT_ANALYZE_ONLY | GFT_NO_JIT |
 *            GFT_KERNEL_TABLE | GFT_KERNEL_WIDE | GFT_NORMALIZED (pass the
 *            combinatorial Laplacian of any bipartite graph: Thm. 2).
 * The plan has no left stages (n_stages = 0), two leaves (E, F) and
 * right_pairs = p.  Transforms run on the CUDA-core kernels (FP32 / FP64;
 * tensor-core precisions return UNSUPPORTED).  Output order as
 * gft_plan_create; signs: the sign rule fixes the sum vector (e_c; f_c) of
 * each unit, and its difference vector (e_c; -f_c) follows.
 * gft_plan_get_leaf_laplacian is UNSUPPORTED for these plans.
 * Errors: INVALID_ARG, NOT_LAPLACIAN, NOT_BIPARTITE, NO_CONVERGENCE, CUDA, OOM.
 */
gft_status gft_plan_create_bipartite(int32_t n, const double* L, const int32_t* side, uint32_t flags,
                                     gft_plan_t* out);

/*
 * Involution search (Sec. V-F): a node involution phi under which L is
 * symmetric (Definition 2, l_ij = l_phi(i)phi(j) within
 * 1e-12*max(1,max|L|), self-loops included), pairing as many nodes as the
 * search finds.  Trees: identical branches with a common or adjacent root
 * are swapped (rooted at the tree's centre, canonical subtree labels);
 * other graphs: depth-first search restricted to equal colours of a
 * colour refinement of the degree list, keeping the involution with the most
 * pairs within max_steps search steps (<= 0: 10^6).
 *  n, L      host, n*n row-major symmetric L (copied).
 *  classes   NULL or n ints: only nodes of equal class may be paired.
 *  phi       host output, n ints (the identity when nothing is found).
 *  pairs     NULL or output: number of pairs (i < phi(i)).
 * Host only; no device work.  Errors: INVALID_ARG, NOT_LAPLACIAN.
 */
gft_status gft_find_involution(int32_t n, const double* L, const int32_t* classes, int64_t max_steps, int32_t* phi,
                               int32_t* pairs);

/*
 * Stages for gft_plan_create found by search: stage s applies
 * gft_find_involution to every block left by stages 0..s-1 (their
 * Laplacians, Eq. 17 stage by stage), pairing only nodes that took part in
 * equally many earlier stages, and lifts the blocks' involutions to the
 * original labels (the recursion at the end of Sec. IV-C).  Stops when no
 * block has a symmetry left or after max_stages (<= 16).
 *  phis      host output, max_stages*n ints (stage-major, original labels).
 *  n_stages  output: stages found (pass to gft_plan_create with phis).
 * Host only.  Errors: INVALID_ARG, NOT_LAPLACIAN.
 */
gft_status gft_search_stages(int32_t n, const double* L, int32_t max_stages, int64_t max_steps, int32_t* phis,
                             int32_t* n_stages);

/* Free a plan and its device memory (NULL is accepted).  The caller must
 * make sure no transform using the plan is still running. */
gft_status gft_plan_destroy(gft_plan_t plan);

typedef struct {
    int32_t n;              /* nodes */
    int32_t n_stages;       /* stages as given, or as found by GFT_SEARCH_STAGES */
    int32_t n_leaves;       /* leaf blocks after all stages (and splitting) */
    int32_t n_pairs;        /* Haar units over all stages */
    int32_t max_leaf;       /* largest leaf size */
    int32_t has_device;     /* 1 if bases are on the device */
    int32_t jacobi_sweeps;  /* most sweeps any leaf needed (0 if analyze-only) */
    uint32_t flags;
    int64_t fast_mults;     /* multiplies per signal: sum of m_k^2 (Sec. V-G) */
    int64_t fast_adds;      /* adds per signal: 2 per Haar unit + sum m_k(m_k-1) */
    int32_t jit;            /* 0: table-driven kernel; 1: plan-specialised kernel with
                               cp.async tiles; 2: plan-specialised with TMA bulk tiles */
    int32_t tile_signals;   /* FP32 forward launch shape chosen by the autotuner: */
    int32_t threads;        /*   signals per tile and threads per block (0 if none) */
    int32_t wide;           /* 1 if FP32 CUDA-core transforms use the wide-leaf kernel */
    int32_t right_pairs;    /* right Haar units (bipartite plans), else 0 */
} gft_plan_info_t;

gft_status gft_plan_get_info(gft_plan_t plan, gft_plan_info_t* info);

/* Haar units of one stage: pairs[2k] = X label, pairs[2k+1] = partner label,
 * in block order.  Pass pairs = NULL to query *count only; otherwise
 * *count is the capacity on entry (in pairs) and the number written on
 * return. */
gft_status gft_plan_get_stage_pairs(gft_plan_t plan, int32_t stage, int32_t* pairs, int32_t* count);

/* Leaf blocks in depth-first order: sizes[n_leaves]; labels[n] holds every
 * leaf's original labels in leaf order, concatenated. */
gft_status gft_plan_get_leaves(gft_plan_t plan, int32_t* sizes, int32_t* labels);

/* Laplacian of one leaf (Eq. 17 applied stage by stage), m*m row-major. */
gft_status gft_plan_get_leaf_laplacian(gft_plan_t plan, int32_t leaf, double* Lk);

/* out_pos[n]: coefficient index of every (leaf, index-in-leaf) entry, in
 * leaf-concatenated order.  Needs device bases (ordering uses eigenvalues). */
gft_status gft_plan_get_output_map(gft_plan_t plan, int32_t* out_pos);

/* Eigenvalues in coefficient order (host, n doubles). */
gft_status gft_plan_eigenvalues(gft_plan_t plan, double* lambda);

/* Full FP64 basis: U host n*n row-major, column j = basis vector of
 * coefficient j, U = B_1 ... B_S diag(U_k) with Eq. 20's stage matrices. */
gft_status gft_plan_basis(gft_plan_t plan, double* U);

/*
 * Forward transform of a batch: y[b, :] = U^T x[b, :] for b < batch.
 * x, y: device, [batch, n] row-major FP32, 16-byte aligned; x == y allowed.
 * precision: GFT_PREC_*; the tensor-core precisions apply to leaves large
 * enough to be a dense contraction and need a plan whose shape the
 * tensor-core kernel supports (UNSUPPORTED otherwise).  batch = 0 is a
 * no-op.  Asynchronous on `stream`.
 */
gft_status gft_plan_forward(gft_plan_t plan, const float* x, float* y, int64_t batch,
                            gft_stream_t stream, uint32_t precision);

/* Inverse transform: x[b, :] = U y[b, :] (B_phi is its own inverse, Sec. III). */
gft_status gft_plan_inverse(gft_plan_t plan, const float* y, float* x, int64_t batch,
                            gft_stream_t stream, uint32_t precision);

/* FP64 forward / inverse (same layout, double).  Only the CUDA-core path. */
gft_status gft_plan_forward_f64(gft_plan_t plan, const double* x, double* y, int64_t batch,
                                gft_stream_t stream);
gft_status gft_plan_inverse_f64(gft_plan_t plan, const double* y, double* x, int64_t batch,
                                gft_stream_t stream);

/*
 * Forward transform of a HOST batch: x_host, y_host are host [batch, n] FP32
 * (pinned memory gives full copy bandwidth).  When both buffers are pinned
 * and mapped into the device address space (cudaHostAlloc / cudaHostRegister,
 * e.g. torch's pin_memory) and FP32 is requested, the transform kernel reads
 * and writes them directly over the host link with no copies; otherwise the
 * plan streams the batch through its own device staging buffers in chunks,
 * overlapping the host-to-device copy, the transform and the device-to-host
 * copy.  Returns when y_host is complete.
 */
gft_status gft_plan_forward_host(gft_plan_t plan, const float* x_host, float* y_host,
                                 int64_t batch, uint32_t precision);

/* Source text of the plan-specialised kernel module (FP32 if f64 == 0,
 * else FP64): pass buf = NULL to query the length (including the NUL). */
gft_status gft_plan_kernel_source(gft_plan_t plan, int32_t f64, char* buf, int64_t* len);

/* Synchronise the plan's last stream and read (and clear) the plan's device
 * error word: 0 = none, else a GFT_ERR_* code a kernel recorded. */
gft_status gft_device_error(gft_plan_t plan, int32_t* code);

/*
 * Mixed batch: many plans, each with its own batch of signals, transformed
 * forward by one CUDA-graph launch, captured on first use and replayed.
 * Plans are routed by leaf width:
 *   - with a tensor-core precision, plans with a leaf of 64 or more nodes:
 *     plans with at most 4096 signals (or leaves of 257..512 nodes) go to
 *     the few-signals tensor-core kernels (signals on the MMA's N axis, up
 *     to 128 per tile; leaves up to 512; two pack launches -- short and long
 *     rows -- and one persistent MMA kernel); the others (leaves up to 256)
 *     to ONE persistent pack kernel and ONE persistent tensor-core kernel
 *     (128 signals per tile) per size class (n <= 256 and n > 256); a timeout
 *     in these kernels is reported in the error word of the plan being
 *     transformed (pack / 128-signal kernel: the class's first plan);
 *   - plans of at most 64 nodes (leaf matrices of at most 2048 entries)
 *     whose entries hold at least 2^19 coefficients in all: ONE persistent
 *     kernel of a module generated and compiled (NVRTC) at creation, with
 *     the straight-line forward code of each such plan (the single-plan
 *     specialised kernel's), over all their (entry, tile) items; unless
 *     GFT_BATCH_NO_JIT;
 *   - the other plans of at most 256 nodes with leaves of at most 64 nodes
 *     and no right Haar units: persistent node-major table-driven kernels,
 *     one launch per size class (n up to 16, 32, 64, 128, 256), tiles of
 *     16..1024 signals, each CTA walking a contiguous, cost-balanced range
 *     of (plan, tile) items with double-buffered tile and program loads;
 *   - the rest with leaves of at most 64 nodes (unless the plan prefers the
 *     wide-leaf kernel): persistent thread-per-signal table-driven kernels,
 *     one launch per size class (row stride n|1 up to 17, 33, 65, 129, 257),
 *     per-plan tile shapes timed at creation;
 *   - leaves of 33..512 nodes otherwise: ONE persistent wide-leaf kernel
 *     over the (plan, tile) items of those plans.
 * Every CUDA-core group computes each output with the same FMA sequence as
 * the plan's own FP32 forward, so their results agree bit for bit.
 * The CUDA-core groups run one after another on the capture stream, the
 * wide-leaf and tensor-core groups on forked streams; all join at the end
 * of the graph.
 *  plans[n_plans]  plans created with device bases; the batch does not own
 *                  them, and they must outlive it.  A plan may appear more
 *                  than once (its entries then run one after another).
 *  batches[n_plans] signals per plan.
 *  flags           precision of the tensor-core leaves: GFT_PREC_FP32 (0:
 *                  CUDA cores only), GFT_PREC_BF16, GFT_PREC_BF16X3,
 *                  GFT_PREC_FP16X3; or'ed with GFT_BATCH_NO_JIT to keep
 *                  every plan off the plan-specialised group.
 * gft_batch_forward: x[i], y[i] device pointers to [batches[i], n_i] FP32
 * (host arrays of n_plans pointers); x[i] != y[i] for tensor-core entries.
 * The captured graph is reused: new pointers are written to the kernels'
 * device descriptors before the replay.
 */
gft_status gft_batch_create(int32_t n_plans, const gft_plan_t* plans, const int64_t* batches,
                            uint32_t flags, gft_batch_t* out);
gft_status gft_batch_forward(gft_batch_t batch, const float* const* x, float* const* y,
                             gft_stream_t stream);
/* Tile configuration of entry i of a CUDA-core group: signals per tile and
 * threads per block (thread-per-signal kernel: 128 threads, a tile chosen by
 * the autotuner; node-major kernel: 256 threads, a power-of-two tile of
 * 16..1024 signals; plan-specialised group: 128 threads, 128..512 signals);
 * 0 for entries routed to the wide-leaf or tensor-core kernels. */
gft_status gft_batch_get_tile(gft_batch_t batch, int32_t i, int32_t* tile, int32_t* threads);
/* Kernel launches of this library in one gft_batch_forward (the nodes of
 * the captured graph that run our kernels). */
gft_status gft_batch_get_launches(gft_batch_t batch, int32_t* launches);
gft_status gft_batch_destroy(gft_batch_t batch);

/*
 * Approximate GFT by layers of Givens rotations (the comparison method of
 * Sec. VI-B: greedy parallel Jacobi layers), alone (n_stages = 0) or after
 * the Haar stages of the symmetric decomposition ("Haar + approximate GFT":
 * the approximation replaces the dense sub-GFTs of the leaves).
 * Build (host, FP64): the stages and leaf Laplacians as gft_plan_create;
 * per leaf, n_layers layers, each pairing nodes greedily by the magnitude of
 * the current off-diagonal entries (largest first, ties by (p, q); entries
 * <= 1e-14*max(1,max|L_k|) count as zero, and a leaf with none left stops)
 * and applying the rotations J(p,q,theta) that zero them, all at once
 * (A <- J^T A J, the symmetric 2x2 Schur rotation); layer t of every leaf
 * runs side by side.  Output order: ascending diagonal of the final A (the
 * approximate eigenvalues), clusters by (leaf, index).  Transform: the units
 * in layer order -- Haar units (x_p, x_q) <- ((x_p + x_q), (x_p - x_q))/sqrt2,
 * rotations (x_p, x_q) <- (c x_p - s x_q, s x_p + c x_q) -- then the
 * permutation; coefficients approximate U^T x.
 *  n, L, n_stages, phi  as gft_plan_create (n <= 1024).
 *  n_layers  Givens layers per leaf, 0..4096.
 *  flags     GFT_SPLIT_COMPONENTS | GFT_ANALYZE_ONLY (no device data).
 * Errors: INVALID_ARG, NOT_LAPLACIAN, NOT_INVOLUTION, BLOCK_LEAK,
 * NOT_SYMMETRIC, UNSUPPORTED, CUDA, OOM.
 */
gft_status gft_approx_create(int32_t n, const double* L, int32_t n_stages, const int32_t* phi, int32_t n_layers,
                             uint32_t flags, gft_approx_t* out);
gft_status gft_approx_destroy(gft_approx_t a);

typedef struct {
    int32_t n;
    int32_t n_haar_layers;  /* leading layers of Haar units (the stages) */
    int32_t n_layers;       /* all layers: Haar, then Givens (a leaf may stop early) */
    int32_t n_units;        /* Haar units + rotations */
    int32_t has_device;
    int32_t tile_signals;   /* signals per CTA tile of the transform kernel */
    int64_t mults;          /* per signal: 4 per rotation, 2 per Haar unit */
    int64_t adds;           /* per signal: 2 per unit */
} gft_approx_info_t;

gft_status gft_approx_get_info(gft_approx_t a, gft_approx_info_t* info);

/* The transform: layer_off[n_layers + 1] (units of layer l are
 * [layer_off[l], layer_off[l+1])), pairs[2 * n_units] (p, q),
 * coef[4 * n_units] (m00, m01, m10, m11: (x_p, x_q) <- (m00 x_p + m01 x_q,
 * m10 x_p + m11 x_q), FP64 as built), perm[n] (coefficient j is node
 * perm[j] after the last layer).  Host outputs sized from get_info. */
gft_status gft_approx_get_units(gft_approx_t a, int32_t* layer_off, int32_t* pairs, double* coef, int32_t* perm);

/* Approximate eigenvalues (host, n doubles) in coefficient order. */
gft_status gft_approx_eigenvalues(gft_approx_t a, double* lambda);

/* U_hat (host n*n row-major, FP64): column j = basis vector of coefficient j. */
gft_status gft_approx_basis(gft_approx_t a, double* U);

/* y[b, :] = U_hat^T x[b, :]: x, y device [batch, n] FP32, 16-byte aligned,
 * x != y.  FP32 arithmetic (units rounded from FP64).  Asynchronous. */
gft_status gft_approx_forward(gft_approx_t a, const float* x, float* y, int64_t batch, gft_stream_t stream);

/*
 * Layered Givens rotations (Eq. 1 and Fig. 1) used as a learned surrogate of
 * a dense GFT: y = G_S ... G_1 x, each stage n/2 rotations on disjoint pairs,
 * (y_p, y_q) = (c x_p - s x_q, s x_p + c x_q) with c = cos(theta), s = sin(theta).
 *  n         even, 2 <= n <= 1024; n_stages 1..64.
 *  pairs     host int32 [n_stages][n/2][2]; each stage a perfect matching, copied.
 */
gft_status gft_givens_create(int32_t n, int32_t n_stages, const int32_t* pairs, gft_givens_t* out);
gft_status gft_givens_destroy(gft_givens_t g);

/* theta: device [n_stages][n/2] FP32.  x, y: device [batch, n] FP32. */
gft_status gft_givens_forward(gft_givens_t g, const float* theta, const float* x, float* y,
                              int64_t batch, gft_stream_t stream);

/*
 * Backward pass: given the forward OUTPUT y and the loss gradient gy, write
 * gx = G_1^T ... G_S^T gy and gtheta[s][k] = sum_b (-g_p y_q + g_q y_p), with
 * stage inputs recovered by inverse rotation (no stored activations).
 * gtheta is overwritten (not accumulated); the sum over the batch is
 * deterministic.  Uses device scratch owned by g.
 */
gft_status gft_givens_backward(gft_givens_t g, const float* theta, const float* y,
                               const float* gy, float* gx, float* gtheta, int64_t batch,
                               gft_stream_t stream);

/*
 * Allocation-free variant of gft_givens_backward (the paper has no
 * counterpart: it is an integration aid).  For callers that cannot allocate
 * device memory once running -- programs whose own pool or fixed budget
 * owns all device memory, real-time loops that must not wait for or risk a
 * failed allocation mid-step, and thin C hosts without an allocator.  It
 * needs no gft_givens_t and calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *  pairs     HOST int32 [n_stages][n/2][2], each stage a perfect matching
 *            (checked; GFT_ERR_INVALID_ARG otherwise), copied every call.
 *  theta     device [n_stages][n/2]; y (forward output), gy, gx: device
 *            [batch, n] FP32, 16-byte aligned; gtheta: device [n_stages][n/2],
 *            overwritten.  Same results as gft_givens_backward (angle sums may
 *            differ in rounding because the CTA count can differ).
 * Scratch: a fixed 4 MiB device array compiled into the library (held on
 * every GPU that loads it until exit) holds the pair table and one row of
 * n_stages*n/2 partial sums per CTA.  A network whose pair table plus one
 * row exceeds 4 MiB is rejected with GFT_ERR_INVALID_ARG (cannot happen
 * within the n and n_stages limits); the CTA count is one per row that fits,
 * a cap the shared-memory limit of the kernel keeps from ever binding.
 * Every call rewrites what it reads, so nothing needs clearing between
 * calls, but all calls share the one array: calls that overlap on the GPU
 * (different streams, or different host threads) race and must be
 * serialised by the caller.  Every call copies `pairs` into the array with
 * cudaMemcpyAsync on `stream`: from pinned memory the copy runs later on the
 * stream, so the table must stay unchanged until then; from pageable memory
 * the driver has staged it when the call returns.  batch = 0 copies the table
 * and zeroes gtheta.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) and keeps it for the life of the
 * process; make that first call before any stream capture (this concerns
 * the look-up only).  After cudaDeviceReset the kept address is stale:
 * restart the process before calling again.
 */
gft_status gft_givens_backward_noalloc(int32_t n, int32_t n_stages, const int32_t* pairs, const float* theta,
                                       const float* y, const float* gy, float* gx, float* gtheta,
                                       int64_t batch, gft_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GFT_H */
