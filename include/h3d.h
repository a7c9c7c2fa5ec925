/*
 * h3d.h -- C ABI of the GB300 HODLR3D library (libh3d.so).
 *
 * HODLR3D (Kandappan, Gujjula & Ambikasaran, arXiv 2307.16303) represents the
 * kernel matrix A_ij = f(|r_i - r_j|), A_ii = 0 (Sec. 3.1, Eq. Laplace3D), of N
 * points in a cube on a uniform octree (Sec. 2.1).  Pairs of same-level boxes
 * that share no boundary or only a vertex are admissible (Definition admh3d) and
 * are stored as low-rank factors found by partially pivoted ACA (Sec. 4.1,
 * Eq. prank); self, edge and face neighbours at the leaf level stay dense and
 * are recomputed on the fly in every product (Alg. 2).
 *
 * Conventions for every entry point:
 *   - Pointers named "device" must be CUDA device (or managed) memory on the
 *     current device; the caller owns them.  Host pointers are plain memory;
 *     page-locked memory makes the copies of h3d_matvec_host asynchronous.
 *   - Point order: x and y are always in the caller's original point order;
 *     the library permutes internally.
 *   - Multi-column vectors are N x nrhs, column-major (column c starts at c*N).
 *   - Element type of x and y is double for H3D_FP64 handles and float for
 *     H3D_FP32 and H3D_FP32_3XTF32 handles.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Products
 *     are stream-ordered and asynchronous; the build synchronises the stream.
 *   - Errors are returned as h3d_status, never by abort.  A device-side error
 *     (for example a point outside the domain) is reported by the call that
 *     detects it; a bounded device wait of an asynchronous product that gave
 *     up leaves H3D_ERR_TIMEOUT in the handle's error word, which the next
 *     call on the handle reports once (and clears).
 *   - A handle may be used by one stream at a time; concurrent calls on one
 *     handle race on its internal scratch buffers.
 */
#ifndef H3D_H
#define H3D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct h3d_handle_s *h3d_handle;

typedef enum {
    H3D_OK = 0,
    H3D_ERR_ARG = 1,       /* invalid argument (null pointer, bad size, unsupported option) */
    H3D_ERR_DOMAIN = 2,    /* a point lies outside the domain cube, or is NaN/Inf          */
    H3D_ERR_OOM = 3,       /* a device allocation failed                                   */
    H3D_ERR_CUDA = 4,      /* a CUDA runtime call or kernel launch failed                  */
    H3D_ERR_ACA_RANK = 5,  /* an admissible block did not reach the tolerance by rank_cap  */
    H3D_ERR_TIMEOUT = 6,   /* a bounded device wait of an earlier product gave up          */
    H3D_ERR_STATE = 7,     /* handle in an unusable state (an earlier call failed)         */
    H3D_ERR_DEPTH = 8      /* more than leaf_size coincident points: depth would exceed 21 */
} h3d_status;

/* Kernel functions f(r) of Sec. 3.1 / Sec. 5.1.  Laplace and Yukawa carry the
 * 1/(4 pi) normalisation; the paper's own 1/r^4 and cos(r)/r are unnormalised. */
typedef enum {
    H3D_LAPLACE = 0,   /* 1 / (4 pi r)                 */
    H3D_YUKAWA = 1,    /* exp(-kappa r) / (4 pi r)     */
    H3D_INV_R4 = 2,    /* 1 / r^4                      */
    H3D_COS_R = 3      /* cos(r) / r                   */
} h3d_kernel;

/* Storage and arithmetic type of the factors, the near field and x / y.
 * ACA pivots, residuals and stopping tests are always FP64.
 *   FP64         FP64 factors and arithmetic on CUDA cores.
 *   FP32         FP32 factors and arithmetic on CUDA cores (products of several
 *                columns in passes of 8 right-hand sides).
 *   FP32_3XTF32  FP32 factors; products of more than 8 columns (leaf_size <=
 *                128) take the factor products to the tensor cores in passes of
 *                32 right-hand sides, each FP32 operand split into two TF32
 *                parts (hi + lo) and the three significant partial products
 *                accumulated in FP32; products of up to 8 columns are those of
 *                FP32.  The default.                                          */
typedef enum {
    H3D_FP64 = 0,
    H3D_FP32 = 1,
    H3D_FP32_3XTF32 = 2
} h3d_precision;

/* Which same-level box pairs are stored as low-rank blocks.  HODLR3D is the
 * paper's format (Def. admh3d); the other two are its comparison formats on the
 * same octree: the H-matrix with the strong condition max(diam) <= eta dist,
 * eta = sqrt(3) (Sec. 2.2, Eq. adm: only pairs sharing no boundary), and HODLR,
 * which compresses every off-diagonal pair (Sec. 2.3).                       */
typedef enum {
    H3D_ADM_HODLR3D = 0,   /* vertex-sharing and well-separated pairs            */
    H3D_ADM_STRONG = 1,    /* well-separated pairs only (H-matrix, eta = sqrt 3) */
    H3D_ADM_WEAK = 2       /* every off-diagonal pair (HODLR)                    */
} h3d_admissibility;

/* What a handle keeps of each admissible block (Sec. 4.1).
 *   FACTORS   the ACA factors U, V (FP32 or FP64): products stream them.
 *   SKELETON  the paper's own storage: the pivots sigma, tau and an LU factorisation
 *             of K(sigma,tau) (FP64, partial pivoting).  Products recompute every
 *             entry of K(sigma,Y) and K(X,tau) in FP64 (their weights carry the
 *             condition of K(sigma,tau), so FP32 entries would not do) and solve
 *             with the LU; memory is O(sum of r^2) instead of O(sum of r (m+n)).
 *             Supports every product call (passes of up to 16 columns, each
 *             entry evaluated once per pass), h3d_energy and h3d_forces;
 *             h3d_matvec_profile returns H3D_ERR_ARG.
 *   SYMMETRIC factors as FACTORS, but every kernel here is symmetric
 *             (K(Y,X) = K(X,Y)^T), so each unordered admissible pair {X, Y} is
 *             compressed once, as the block whose target box has the smaller
 *             index; the block (Y, X) is its transpose, V U^T, with the swapped
 *             pivots (tau, sigma) (Eq. prank transposed).  The operator is then
 *             symmetric, and h3d_matvec_T runs the forward product.  Pairs whose
 *             factors fit in shared memory (most of the deep levels) are stored
 *             once and read once per product for both directions; the others
 *             are stored for both orders in the FACTORS layout.  The fused
 *             pairs' two contributions are summed with FP64 atomic additions, so
 *             results may differ in the last bits from run to run.  FP32 handles
 *             compute products of more than one column in passes of 8 (no
 *             tensor-core path).  h3d_export_pivots returns the mirrors' swapped
 *             pivots; h3d_import_pivots requires them (H3D_ERR_ARG otherwise).
 *             Batches take the graph form.                                   */
typedef enum {
    H3D_STORE_FACTORS = 0,
    H3D_STORE_SKELETON = 1,
    H3D_STORE_SYMMETRIC = 2
} h3d_storage;

typedef struct {
    int precision;          /* h3d_precision, default H3D_FP32_3XTF32                   */
    double kappa;           /* Yukawa decay, default 1.0                                 */
    int rank_cap;           /* largest ACA rank per block, 1..512, default 512           */
    double lo[3];           /* lower corner of the domain cube, default (-1,-1,-1)       */
    double side;            /* edge length of the domain cube, default 2.0               */
    int64_t workspace_bytes;/* device scratch budget for the build; 0 = automatic, >= 0  */
    int admissibility;      /* h3d_admissibility, default H3D_ADM_HODLR3D                */
    int storage;            /* h3d_storage, default H3D_STORE_FACTORS                    */
} h3d_options;

/* Fill *opt with the defaults listed above. */
void h3d_default_options(h3d_options *opt);

/* Alg. 1 (InitializeHODLR3D): build the octree, the interaction and near lists
 * and the ACA factors of every admissible block.
 *   points    device, N x 3 row-major FP64 coordinates (x0,y0,z0,x1,...).  Not
 *             retained: the handle keeps its own sorted copy.
 *   N         number of points, 1 <= N < 2^31.
 *   kernel    h3d_kernel.
 *   leaf_size N_max of Sec. 2.1: the depth L is the smallest level at which no
 *             box holds more than leaf_size points; 1..512.
 *   tol       ACA tolerance epsilon of Alg. 1 (>= 0; 0 asks for full rank).
 *   opt       NULL for defaults.
 *   stream    stream for all device work; synchronised before return.
 *   out       receives the handle; untouched on error.
 * Errors: H3D_ERR_ARG, H3D_ERR_DOMAIN, H3D_ERR_DEPTH, H3D_ERR_ACA_RANK,
 *         H3D_ERR_OOM, H3D_ERR_CUDA.  On error every allocation is released.  */
h3d_status h3d_build(const double *points, int64_t N, h3d_kernel kernel, int leaf_size,
                     double tol, const h3d_options *opt, void *stream, h3d_handle *out);

/* Alg. 2 (MatVec): y = A~ x, the dense near field recomputed on the fly plus the
 * low-rank blocks of every level.
 *   x  device, N x nrhs in the caller's order (read only).
 *   y  device, N x nrhs, overwritten (not accumulated).  Must not alias x.
 *   nrhs >= 1.  Several right-hand sides share each pass over the factors (up
 *   to 8 per pass, or 32 for H3D_FP32_3XTF32 handles with leaf_size <= 128).
 * Enqueues kernels on `stream` and returns.  Allocates nothing, except that the
 * first call with nrhs > 8 on an H3D_FP32_3XTF32 handle allocates (and keeps)
 * the scratch of the 32-column passes after synchronising `stream`; make that
 * first call before capturing products into a CUDA graph.                    */
h3d_status h3d_matvec(h3d_handle h, const void *x, void *y, int nrhs, void *stream);

/* y = A~^T x: the same blocks with the roles of the two factors exchanged (the
 * compressed operator is not exactly symmetric because every ordered pair is
 * compressed on its own, as Alg. 1 does; with H3D_STORE_SYMMETRIC it is, and
 * this runs the forward product).  Arguments as h3d_matvec.                  */
h3d_status h3d_matvec_T(h3d_handle h, const void *x, void *y, int nrhs, void *stream);

/* Energy of charges q and its gradient (differentiation of the product):
 *   E = 1/2 q^T A~ q,   grad = dE/dq = 1/2 (A~ + A~^T) q
 * with A~ the operator of h3d_matvec (Alg. 2); both products are taken because
 * A~ is not exactly symmetric (Alg. 1 compresses every ordered pair on its own;
 * with H3D_STORE_SYMMETRIC it is, and one product gives both).
 *   q     device, N values in the caller's order (read only).
 *   E     device, one double: the energy, reduced in FP64 in a fixed order.
 *   grad  device, N values (element type of the handle), overwritten; NULL skips
 *         the transpose product and the gradient.  Must not alias q.
 * Enqueues on `stream`; the first call allocates (and keeps) 2N values of
 * scratch after synchronising `stream`.                                       */
h3d_status h3d_energy(h3d_handle h, const void *q, double *E, void *grad, void *stream);

/* Forces on the points for the same energy, F = -dE/dp, with the ACA pivots of
 * the build frozen: the near blocks are exact kernel entries and each
 * admissible block (X, Y) is the cross form K(X,tau) K(sigma,tau)^{-1} K(sigma,Y)
 * of its pivots (Sec. 4.1, Eq. prank), so E is the energy of the paper's
 * representation (it equals that of h3d_energy up to rounding times the
 * condition of K(sigma,tau)).  Kernel entries and their gradients are
 * recomputed (nothing is stored): the admissible blocks to ~1e-12 or better
 * (their weights carry the condition of K(sigma,tau)): in FP64 for FP64
 * handles, in float-float on the FP32 pipes for FP32 handles of the Laplace
 * and 1/r^4 kernels, in FP64 for the other FP32 handles; the near field in the
 * handle's precision; K(sigma,tau) is factored in FP64 with partial pivoting.
 * Supported for every kernel of h3d_kernel and every storage.
 *   q  device, N charges in the caller's order (element type of the handle).
 *   E  device, one double: the energy.
 *   F  device, N x 3 doubles, row-major, the caller's order; overwritten.
 * Enqueues on `stream`; the first call allocates (and keeps) O(N) doubles and a
 * scratch of max_rank^2 doubles per CTA after synchronising `stream`.          */
h3d_status h3d_forces(h3d_handle h, const void *q, double *E, double *F, void *stream);

/* ---- Batches of independent operators (many point clouds) ------------------
 * A batch runs the products y_i = A~_i x_i of several handles (one right-hand
 * side each; Alg. 2 for every operator) in one of two forms:
 *   persistent  ONE launch of a persistent kernel whose CTAs take work items of
 *               every operator from a device queue (permute, gather,
 *               near-field, reduce and leaf items; an item waits, with a
 *               bounded wait, until the items it reads are complete), replayed
 *               as a CUDA graph together with the reset of the queue.  Available when every handle
 *               stores factors (H3D_STORE_FACTORS) and all are FP64, or all
 *               FP32 or FP32_3XTF32 (the two may be mixed: a batch runs one
 *               column per handle); it is then the default.
 *   graph       every handle's own product (the kernels of h3d_matvec) captured
 *               once into a CUDA graph on `branches` concurrent streams, clouds
 *               assigned longest first to the least loaded stream; later calls
 *               with the same vectors replay it (new vectors re-capture).
 * The handles must be distinct (H3D_ERR_ARG otherwise), must outlive the batch
 * and must not be used elsewhere while a batch product is in flight, and
 * h3d_import_pivots on a member invalidates the batch (free and re-create it).
 * A wait that runs out in the persistent kernel leaves H3D_ERR_TIMEOUT in
 * that handle's error word (reported once by the next call on the batch or
 * the handle).
 *   handles  host array of `count` built handles.
 *   x, y     host arrays of `count` device pointers: x[i], y[i] are N_i values
 *            of handle i's element type (caller's order); y overwritten.  In the
 *            persistent form new pointers are copied to the device, in stream
 *            order, by the call that first uses them.
 * h3d_batch_tune times (three runs after a warm-up, CUDA events on `stream`)
 * the graph form with 1, 2, 4, ... branches (up to 32 and the number of
 * handles) and, when available, the persistent form: first one item shape for
 * every operator -- leaves per item (near, leaf) in {(4,1), (4,2), (8,4)} --
 * with queue orders phase-major or pipelined over operators (lag 2 or 8) and
 * the most resident CTAs per SM or one fewer (default: (4,2), lag 0, the
 * most); then, from the best of those, the item shape of each (size, rank)
 * bucket of operators in turn (N < 2^15, < 2^17 or larger; largest rank <= 96
 * or larger) among (2,1), (4,1), (4,2), (8,2), (8,4), (16,4).  It keeps the
 * fastest form and reports in *branches_out (may be NULL) the branch count, or
 * 0 for the persistent form.  It synchronises `stream`.
 * h3d_batch_groups writes the persistent form's leaves per near-field item and
 * per leaf item of every operator (host arrays of `count` ints, either may be
 * NULL); H3D_ERR_ARG without a persistent form.
 * h3d_batch_configure selects the form (persistent != 0: the persistent kernel;
 * H3D_ERR_ARG if it is not available) and the persistent form's settings: CTAs
 * per SM of its grid (capped at the occupancy limit), leaves per near-field
 * item and per leaf item, and the queue order (lag 0: phase-major; d > 0:
 * pipelined over operators); 0 (-1 for lag) keeps the current value.  The
 * settings change who computes an item and when, never how: the persistent
 * form's results are the same bits for every setting.  h3d_batch_info reports
 * the form in use (*persistent: 1 persistent, 0 graph, -1 graph and persistent
 * unavailable),
 * the CTAs per SM of the persistent form and the branch count of the graph
 * form; any pointer may be NULL.                                              */
typedef struct h3d_batch_s *h3d_batch;
h3d_status h3d_batch_create(const h3d_handle *handles, int count, h3d_batch *out);
h3d_status h3d_batch_matvec(h3d_batch b, const void *const *x, void *const *y, void *stream);
h3d_status h3d_batch_tune(h3d_batch b, const void *const *x, void *const *y, void *stream, int *branches_out);
h3d_status h3d_batch_configure(h3d_batch b, int persistent, int ctas_per_sm, int near_group, int leaf_group,
                               int lag);
h3d_status h3d_batch_info(h3d_batch b, int *persistent, int *ctas_per_sm, int *branches);
h3d_status h3d_batch_groups(h3d_batch b, int *near_groups, int *leaf_groups);

/* Bound of every wait of the persistent kernel on the completion counters of
 * the items it depends on, in nanoseconds of the GPU's global timer
 * (default 2e9, i.e. 2 s; 1e3 <= ns <= 6e10, else H3D_ERR_ARG).  A wait that
 * runs out stops the launch: the handle of the waiting item gets
 * H3D_ERR_TIMEOUT, the results of that product are not valid, and the handles
 * and the batch stay usable.  Without a persistent form it is H3D_OK and has
 * no effect.                                                                  */
h3d_status h3d_batch_set_wait_limit(h3d_batch b, int64_t ns);

/* The persistent form's work queue (for tests and inspection).
 * h3d_batch_get_queue: *count = items in the queue; items (host, 4 ints per
 * item as in h3d_batch_queue, capacity `cap` items; NULL: only count).
 * h3d_batch_set_queue: run the persistent kernel on the caller's `count` items
 * (host, same format) instead; each item must name an operator of the batch
 * and lie inside its work (H3D_ERR_ARG otherwise), but nothing checks that
 * every item comes after the items it waits for: a queue that breaks that
 * order ends in the bounded waits (H3D_ERR_TIMEOUT).  items = NULL returns to
 * the queue of the current settings.  H3D_ERR_ARG without a persistent form. */
h3d_status h3d_batch_get_queue(h3d_batch b, int *items, int64_t cap, int64_t *count);
h3d_status h3d_batch_set_queue(h3d_batch b, const int *items, int64_t count);

/* The persistent batch form's work queue for operators of the given sizes
 * (host only, no device work; for tests and inspection).  Operator o has
 * n_points[o] >= 1 points, n_gather[o] gather tasks, n_split[o] split source
 * boxes and n_leaves[o] >= 1 leaves; near_group, leaf_group >= 1 and lag >= 0
 * as in h3d_batch_configure.  items (host, 4 ints per item, capacity `cap`
 * items; NULL: only count) receives (operator, kind, first, count) with kind 0
 * gather task, 1 near-field leaf run, 2 split-box reduction, 3 leaf run,
 * 4 permute chunk (first point; count unused); *count the number of items.
 * H3D_ERR_ARG on bad sizes or a capacity below the count.  Every item comes
 * after the items it waits for: an operator's permute chunks before its gather
 * and near-field items, its gathers before its reductions, and its gathers,
 * reductions and near-field runs before its leaf runs.                       */
h3d_status h3d_batch_queue(int nops, const int64_t *n_points, const int *n_gather, const int *n_split,
                           const int *n_leaves, int near_group, int leaf_group, int lag, int *items, int64_t cap,
                           int64_t *count);
h3d_status h3d_batch_free(h3d_batch b);

/* h3d_matvec with HOST x and y: copies x to the device, runs the product and
 * copies y back, all on `stream`, then synchronises the stream.  Device staging
 * buffers are allocated on the first call (and grown if nrhs grows) and kept by
 * the handle.                                                                 */
h3d_status h3d_matvec_host(h3d_handle h, const void *x_host, void *y_host, int nrhs, void *stream);

/* Release every device allocation of the handle.  h3d_free(NULL) is H3D_OK.
 * Synchronises the device before freeing.                                    */
h3d_status h3d_free(h3d_handle h);

/* Static English text for a status code. */
const char *h3d_status_string(h3d_status s);

/* Sizes and counts of a built handle (Table "ResultsNotations" quantities). */
typedef struct {
    int64_t N;
    int depth;                 /* L                                                 */
    int precision, kernel, leaf_size;
    double tol;
    int64_t n_boxes;           /* non-empty boxes, all levels                       */
    int64_t n_leaves;
    int64_t n_blocks;          /* admissible (low-rank) blocks, all levels          */
    int64_t n_vertex_blocks;   /* of which vertex-sharing                           */
    int64_t n_near;            /* dense self/edge/face leaf pairs                   */
    int max_rank;
    int64_t sum_rank;
    int64_t factor_entries;    /* sum over blocks of r (m + n) (symmetric storage:
                                  stored entries, fused pairs counted once)         */
    int64_t u_entries;         /* sum over blocks of r m (target-side factors)      */
    int64_t v_entries;         /* sum over blocks of r n (source-side factors)      */
    int64_t factor_bytes;      /* stored factor bytes including padding             */
    int64_t near_interactions; /* sum over near pairs of m * n                      */
    int64_t device_bytes;      /* all device memory held by the handle              */
    double build_ms;
} h3d_stats;

h3d_status h3d_get_stats(h3d_handle h, h3d_stats *s);

/* h3d_matvec with per-phase timing, for profiling: the same kernels on `stream`,
 * bracketed by CUDA events; synchronises the stream and writes the summed
 * durations in milliseconds over all right-hand sides to phase_ms[0..nphase):
 *   0 permutation of x, 1 source-side gather V^T x, 2 reduction of split
 *   gathers, 3 per-leaf kernel (near field + target-side U t + permutation of y).
 * Symmetric storage: 1 is the fused pairs' kernel (both directions, on a stream
 *   of its own beside the other pairs' gather) and 2 the rest of that gather
 *   with its reduction and the addition of the fused contributions to the near
 *   field.
 * phase_ms: host, nphase >= 1 (at most 4 entries are written).              */
h3d_status h3d_matvec_profile(h3d_handle h, const void *x, void *y, int nrhs, void *stream,
                              float *phase_ms, int nphase);

/* Diagnostics (host outputs; sizes from h3d_get_stats; used by the tests).
 * Tree: perm[s] = original index of the s-th point in Morton order; keys[s] its
 * 63-bit Morton key; nbox[l] (l = 0..L) non-empty boxes per level; box_key /
 * box_start / box_end per box, levels concatenated in order, boxes in Morton
 * order within a level (box_key is the 3l-bit Morton prefix).                */
h3d_status h3d_export_tree(h3d_handle h, int64_t *perm, uint64_t *keys, int *nbox,
                           uint64_t *box_key, int64_t *box_start, int64_t *box_end);

/* Lists: admissible blocks in (level, target, source) order with level-local
 * box indices and class 1 = face, 2 = edge (weak admissibility only), 3 =
 * vertex, 4 = well separated; near pairs (leaf level) in (target, source) order
 * with class 0 = self, 1 = face, 2 = edge, 3 = vertex (strong only).        */
h3d_status h3d_export_lists(h3d_handle h, int *blk_level, int *blk_tgt, int *blk_src, int *blk_cls,
                            int *near_tgt, int *near_src, int *near_cls);

/* ACA ranks (per block) and pivots (concatenated in block order): sigma are
 * row indices local to the target box, tau column indices local to the source. */
h3d_status h3d_export_pivots(h3d_handle h, int *rank, int *sigma, int *tau);

/* Re-form the handle from given ACA pivots (Sec. 4.1, Eq. prank: a block is
 * determined by its pivot rows sigma and columns tau): the same tree and lists,
 * the caller's ranks and pivots, and the factors (or, for skeleton storage,
 * the LU of K(sigma,tau)) formed from them by the ACA recurrences without the
 * pivot search.  Used to compare against pivots found elsewhere (for example
 * by an independent CPU search) and to restore pivots saved earlier.
 *   rank, sigma, tau  host, in the format of h3d_export_pivots; 0 <= rank[b] <=
 *          min(m_b, n_b, rank_cap), indices inside the block, no row or column
 *          twice in one block; with H3D_STORE_SYMMETRIC every mirror block
 *          carries its primary's rank and swapped pivots; otherwise
 *          H3D_ERR_ARG.  Pivots that ACA could not have chosen (a vanishing
 *          residual at a pivot) give non-finite factors.
 * Builds the replacement first (synchronising `stream` and the device) and
 * swaps it in only on success; on error the handle is unchanged.  Batches that
 * hold the handle must be re-created afterwards.                              */
h3d_status h3d_import_pivots(h3d_handle h, const int *rank, const int *sigma, const int *tau, void *stream);

/* Move the points: new coordinates for the same N points, keeping the build's
 * tree, lists, ranks and pivots (frozen) and re-forming the factors (or the LU
 * of K(sigma,tau)) from them at the new positions.  The operator is then the
 * function of the positions that h3d_forces differentiates; points may leave
 * their boxes (nothing is re-sorted), at the cost of accuracy if they move far.
 *   points  device, N x 3 row-major FP64, the caller's order (read only).
 * Coordinates equal to the current ones bit for bit cost one comparison pass
 * and change nothing.  H3D_ERR_DOMAIN (handle unchanged) for a non-finite
 * coordinate.  Synchronises `stream`.                                        */
h3d_status h3d_set_points(h3d_handle h, const double *points, void *stream);

/* Test hook: the next `after` device allocations made by the library succeed
 * and the one after them fails as if the device were out of memory (the call
 * that makes it returns H3D_ERR_OOM and releases what it allocated); after < 0
 * switches the injection off.  Process-wide, not thread-safe.                */
void h3d_debug_fail_alloc(int64_t after);

/* ---- Morton order without allocation (the paper has no counterpart) --------
 * For callers that cannot allocate device memory (a host application that owns
 * a fixed memory pool, a plugin that only receives pre-allocated buffers): the
 * Morton keys and the stable Morton order of N points -- what the first two
 * steps of h3d_build compute -- using only a fixed scratch area of
 * H3D_NOALLOC_SCRATCH_BYTES that is a static device array inside the library.
 * The call itself allocates nothing (no cudaMalloc, cudaFree or allocating
 * library routine).
 *   points    device, N x 3 row-major FP64 (read only).
 *   N         1 <= N <= H3D_NOALLOC_MAX_POINTS; larger N is rejected with
 *             H3D_ERR_ARG (the scratch area has a fixed size).
 *   lo, side  host; the domain cube [lo, lo + side]^3 (lo: 3 doubles).
 *   keys_out  device, N uint64: the sorted 63-bit keys.
 *   perm_out  device, N int32: perm_out[s] = original index of the s-th point.
 *   stream    stream for all work; synchronised before return (to report a
 *             point outside the cube as H3D_ERR_DOMAIN).
 * The scratch array is held by every GPU that loads the library until the
 * process exits and is shared by all calls: calls that overlap on the GPU race
 * and must be serialised by the caller.  The first call on a device resolves
 * the array's device address.  Every call synchronises its stream, so it must
 * not be made while that stream is being captured into a CUDA graph.         */
#define H3D_NOALLOC_MAX_POINTS (1 << 20)
#define H3D_NOALLOC_SCRATCH_BYTES (14 << 20)
h3d_status h3d_morton_order_noalloc(const double *points, int64_t N, const double *lo, double side,
                                    uint64_t *keys_out, int *perm_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* H3D_H */
