// h3d_internal.cuh -- shared declarations of the CUDA HODLR3D library.
//
// Data layout in HBM (all indices refer to points in Morton order):
//   points     px/py/pz: FP64 SoA, sorted; ploc / ploc_lo: float4 per point,
//              the offset from the centre of its leaf box as hi + lo FP32
//              (near field in FP32).
//   boxes      all non-empty boxes of all levels, level-major, Morton order
//              inside a level; index g is "global", g - box_off[l] "level-local".
//   blocks     admissible pairs (target X, source Y) of every level in
//              (level, target, source) order.
//   U factors  target side, per box A at level l: one panel per leaf Z under A,
//              panel = ld_Z x R_A column-major (ld_Z = m_Z rounded up to the
//              vector width), R_A = sum of the ranks of A's blocks.  A leaf
//              task reads one contiguous panel per level.
//   V factors  source side, per box Y: n_Y x ldv_Y row-major, ldv_Y = R'_Y
//              rounded up, R'_Y = sum of ranks of the blocks whose source is Y.
//   t          per block b, r_b entries at tofs_b (target-major order), so the
//              coefficients of all blocks of a target box are contiguous.
//   symmetric  (H3D_STORE_SYMMETRIC) each unordered pair {X, Y} is compressed
//              once, as the block whose target has the smaller index.  Pairs
//              whose factors fit one shared-memory stage ("fused" set) are kept
//              once, block-major in symF: U (ldm x r) then V (ldn x r), both
//              column-major with leading dimensions = 2 (mod 4), blocks packed into
//              16-byte aligned groups of at most one stage.  The other pairs are
//              kept in the U / V layout above for both orders, the mirror (Y, X)
//              holding the transposed factors; the layout counts only their
//              ranks (lrank).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <initializer_list>
#include <vector>

#include "../../include/h3d.h"

namespace h3d {

constexpr int kMaxDepth = 21;
constexpr int kMaxLeaf = 512;
constexpr int kMaxRank = 512;

// 1 / (4 pi) to more digits than a double holds.
#define H3D_INV4PI 0.0795774715459476678844418816863

// ----------------------------------------------------------------------------
// error handling
struct Error {
    h3d_status st;
};

#define H3D_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e__ = (call);                                                        \
        if (e__ != cudaSuccess) {                                                        \
            if (getenv("H3D_DEBUG"))                                                     \
                fprintf(stderr, "h3d: %s failed at %s:%d: %s\n", #call, __FILE__, __LINE__, \
                        cudaGetErrorString(e__));                                        \
            throw ::h3d::Error{e__ == cudaErrorMemoryAllocation ? H3D_ERR_OOM : H3D_ERR_CUDA}; \
        }                                                                                \
    } while (0)

#define H3D_LAUNCH_CHECK() H3D_CUDA(cudaGetLastError())

inline void fail(h3d_status st) { throw Error{st}; }

// Device allocation owned by the handle.
struct DevMem {
    void *p = nullptr;
    size_t bytes = 0;
};

// Allocation-failure injection for tests (h3d_debug_fail_alloc): when >= 0,
// the number of device allocations that still succeed before one fails.
int64_t &fail_alloc_countdown();

class Arena {
  public:
    ~Arena() { release(); }
    void *alloc(size_t bytes) {
        if (bytes == 0) bytes = 16;
        int64_t &cd = fail_alloc_countdown();
        if (cd == 0) {
            cd = -1;
            fail(H3D_ERR_OOM);
        }
        if (cd > 0) --cd;
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(H3D_ERR_OOM);
        }
        blocks_.push_back({p, bytes});
        total_ += bytes;
        return p;
    }
    template <class T>
    T *get(size_t n) { return static_cast<T *>(alloc(n * sizeof(T))); }
    void free_one(void *p) {
        for (size_t i = 0; i < blocks_.size(); ++i)
            if (blocks_[i].p == p) {
                cudaFree(p);
                total_ -= blocks_[i].bytes;
                blocks_.erase(blocks_.begin() + (long)i);
                return;
            }
    }
    void release() {
        for (auto &b : blocks_) cudaFree(b.p);
        blocks_.clear();
        total_ = 0;
    }
    size_t total() const { return total_; }

  private:
    std::vector<DevMem> blocks_;
    size_t total_ = 0;
};

// Scratch a call allocates on first use: every request is made, or, if one
// fails, the ones already made are released and the error is passed on (so a
// later call never finds the scratch half allocated).
struct AllocReq {
    void **dst;
    size_t bytes;
};
inline void alloc_all(Arena &m, std::initializer_list<AllocReq> req) {
    std::vector<void *> got;
    try {
        for (const AllocReq &r : req) got.push_back(m.alloc(r.bytes));
    } catch (...) {
        for (void *p : got) m.free_one(p);
        throw;
    }
    size_t i = 0;
    for (const AllocReq &r : req) *r.dst = got[i++];
}

// ----------------------------------------------------------------------------
// the handle
// One tensor-core gather work item: rows [r0, r0 + nrows) of source box Y's V
// factor, columns [c_lo, c_lo + 128), against 32 right-hand sides.  The V tile is
// read through box Y's 2-D TMA tensor map.
struct TcGatherItem {
    int64_t x;                // first row of the permuted right-hand sides
    int64_t o;                // first output row: map_v offset (to t) or partial row (to partial)
    int tmap;                 // tensor map of the box's V factor
    int c_lo, r0;             // first column and row (within the box) of the tile
    int nrows, ncols, to_t;   // rows, valid columns, output kind
};

// Symmetric storage: one fused pair (offsets in elements of the factor type) and
// one group of fused pairs that a single bulk copy brings into shared memory.
struct SymBlk {
    int64_t off;              // U at off, V at off + r * ldm (in symF)
    int xs, ys, m, n, r;      // first sorted point and size of X and Y, rank
    int ldm, ldn;             // leading dimensions (>= m, n, = 2 mod 4: sym_ld)
    int pad;
};
struct SymGroup {
    int64_t off;              // first element (16-byte aligned)
    int bytes;                // multiple of 16, at most one stage
    int b0, nb;               // SymBlk range
    int big;                  // one pair taken by the whole CTA (else one warp per pair)
};
// Leading dimension of a fused pair's factor: the smallest ld >= m with
// ld = 2 (mod 4).  Columns then start 8 bytes aligned (FP32 pairs of rows load
// as one float2), and both the lanes' column walks (addresses k ld) and their
// row walks touch distinct banks: ld / 2 is odd.
__host__ __device__ inline int sym_ld(int m) {
    int l = (m + 1) & ~1;
    if ((l & 3) == 0) l += 2;
    return l;
}
constexpr int kSymStageF32 = 80 * 1024;   // stage bytes (FP32 / FP64 handles); two stages per CTA
constexpr int kSymStageF64 = 64 * 1024;
constexpr int kSymSmallR = 64;            // a warp takes a pair of rank <= 64 and at most
constexpr int kSymSmallElems = 12288;     // this many factor entries; larger ones a CTA
constexpr int kSymMaxR = 256;             // largest rank of a fused pair
constexpr int kSymGroupPairs = 16;        // small pairs per group (one per warp)

struct Handle {
    // parameters
    int64_t N = 0;
    int kernel = H3D_LAPLACE, prec = H3D_FP32, leaf_size = 0, rank_cap = kMaxRank, adm = H3D_ADM_HODLR3D;
    int storage = H3D_STORE_FACTORS;
    bool tf32 = false;            // H3D_FP32_3XTF32: products of more than 8 columns on the tensor cores
    int64_t budget = 0;           // build workspace budget (h3d_options.workspace_bytes)
    // skeleton storage: per block the LU of K(sigma,tau) (row-major, L unit lower,
    // at lu_off[b]) and its row order (at piv_off[b]); product scratch per block
    double *lu = nullptr;
    int64_t *lu_off = nullptr;                    // nblk + 1
    int64_t lu_off_total = 0;                     // sum of r^2
    int *lu_piv = nullptr;
    double *skel_s = nullptr, *skel_c = nullptr;  // K(sigma,Y) X and K(sigma,tau)^{-1} of it, 16 per pivot
    void *skel_xs = nullptr, *skel_near = nullptr; // pass columns: permuted x point-major, near field
    void *skel_xmr = nullptr, *skel_nmr = nullptr; // blocks of 8 columns for the multi-column near field
    int skel_nq = 16;                             // columns per skeleton pass (memory-bound choice)
    int64_t *skel_src_ptr = nullptr, *skel_src_order = nullptr;   // blocks by source box (transpose)
    int *skel_next = nullptr;                     // next block of the source-side pass (work queue head)
    // FP32 skeleton handles of a kernel that float-float evaluates (Laplace,
    // 1/r^4): coordinates as float-float offsets from the domain centre
    float4 *sffh = nullptr, *sffl = nullptr;
    // large blocks of the skeleton products: (block, pivot) items, per-block slot, pivot sums
    int2 *skel_big = nullptr;
    int64_t skel_nbig = 0, *skel_bigpo = nullptr;
    double *skel_sbig = nullptr;
    double tol = 0, kappa = 1.0, lo[3] = {-1, -1, -1}, side = 2.0;
    int L = 0;
    // symmetric storage: per block its rank in the U / V layout (0 for fused
    // pairs; the ranks themselves elsewhere), the fused pairs and their groups
    int *lrank = nullptr;
    int nsym = 0, nsym_grp = 0;
    SymBlk *sym_blk = nullptr;
    SymGroup *sym_grp = nullptr;
    int *sym_slot = nullptr;                      // per block: fused slot, or -1 (mirrors too)
    std::vector<int> sym_slot_h;                  // host copy
    void *symF = nullptr;
    int64_t sym_elems = 0;                        // stored entries of symF (with padding)
    int64_t sym_entries = 0;                      // sum over fused pairs of r (m + n)
    double *sym_acc = nullptr;                    // fused contributions, N x 8 doubles (Morton order)
    bool symmetric() const { return storage == H3D_STORE_SYMMETRIC; }

    Arena mem;          // everything the handle keeps
    int *d_err = nullptr;
    // error word of the product kernels in mapped host memory: a kernel whose
    // bounded wait gave up stores a status there, the next call reports it
    int *h_async_err = nullptr, *d_async_err = nullptr;
    // second stream for the near field, and the fork / join events
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // symmetric storage: the fused pairs' kernel on a stream of its own, beside
    // the other pairs' gather (it is latency-bound and leaves HBM bandwidth free)
    cudaStream_t sym_stream = nullptr;
    cudaEvent_t ev_sym_fork = nullptr, ev_sym_join = nullptr;
    void *nearbuf = nullptr;                      // near-field result, Morton order (N)
    // multi-RHS scratch: blocks of 8 columns, point-major
    void *xs_mr = nullptr, *nearbuf_mr = nullptr, *t_mr = nullptr, *partial_mr = nullptr;
    // 32-column FP32 scratch, allocated by the first product with more than 8 columns
    void *xs_w = nullptr, *nearbuf_w = nullptr, *t_w = nullptr, *partial_w = nullptr;
    // tensor-core (32-column) work lists, resolved at plan time
    int ntc_items = 0;                            // gather: (task, block of 128 columns)
    struct TcGatherItem *tc_items = nullptr;
    int nsplit_w = 0;                             // gather: boxes split into row tasks (32-column path)
    int *split_box_w = nullptr, *split_ntask_w = nullptr;
    int max_rv_split_w = 0;                       // widest split box (columns)
    int64_t *split_pbase_w = nullptr;
    int64_t partial_elems_w = 0;
    void *tc_tmaps = nullptr;                     // gather: one 2-D tensor map (CUtensorMap) per source box
    int ntc_tiles = 0;                            // far field: sibling leaves packed into 128 rows
    int2 *tc_tiles = nullptr;                     // (first leaf, number of leaves)
    ~Handle() {
        if (side_stream) cudaStreamSynchronize(side_stream);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side_stream) cudaStreamDestroy(side_stream);
        if (sym_stream) cudaStreamSynchronize(sym_stream);
        if (ev_sym_fork) cudaEventDestroy(ev_sym_fork);
        if (ev_sym_join) cudaEventDestroy(ev_sym_join);
        if (sym_stream) cudaStreamDestroy(sym_stream);
        if (h_async_err) cudaFreeHost(h_async_err);
    }

    // points
    double *px = nullptr, *py = nullptr, *pz = nullptr;
    float4 *ploc = nullptr, *ploc_lo = nullptr;
    int *perm = nullptr;         // sorted position -> original index
    uint64_t *keys = nullptr;    // sorted keys

    // boxes
    int nbox[kMaxDepth + 1] = {0};
    int64_t box_off[kMaxDepth + 2] = {0};
    int64_t n_boxes = 0;
    uint64_t *box_key = nullptr;
    int *box_start = nullptr, *box_end = nullptr, *box_parent = nullptr;
    int *box_leaf_lo = nullptr, *box_leaf_hi = nullptr;   // leaf (level-local) range under a box
    int nleaf = 0;
    int *leaf_anc = nullptr;     // [(l-1) * nleaf + z] global ancestor at level l (l = 1..L)
    int *point_leaf = nullptr;   // sorted point -> level-local leaf index

    // blocks (admissible, all levels)
    int64_t nblk = 0;
    int64_t blk_off[kMaxDepth + 2] = {0};
    int *blk_tgt = nullptr, *blk_src = nullptr;  // global box indices
    unsigned char *blk_cls = nullptr, *blk_lev = nullptr;
    int *blk_partner = nullptr;                   // index of the transposed block
    int64_t *tgt_ptr = nullptr;                   // per global box: first block with this target (n_boxes + 1)

    // near lists (leaf level)
    int64_t nnear = 0;
    int *near_ptr = nullptr;                      // per leaf, nleaf + 1
    int *near_src = nullptr;                      // level-local leaf index
    unsigned char *near_cls = nullptr;
    unsigned char *near_dir = nullptr;            // packed offset (dx+1)*9+(dy+1)*3+(dz+1)

    // ranks and pivots
    int *rank = nullptr;
    int64_t *piv_off = nullptr;                   // nblk + 1
    int *sigma = nullptr, *tau = nullptr;
    int64_t sum_rank = 0;
    int max_rank = 0;

    // factor layout
    int *R = nullptr;                             // per box: target-side columns
    int64_t *tbase = nullptr;                     // per box: first t entry of its blocks
    int64_t *ubase = nullptr;                     // per box: U element offset
    int *Rv = nullptr, *ldv = nullptr;            // per box: source-side columns and row stride
    int64_t *vbase = nullptr;                     // per box: V element offset
    int64_t *vcol0 = nullptr;                     // per box: first global V column
    int *cu = nullptr, *cv = nullptr;             // per block: column offset in target / source box
    int64_t *tofs = nullptr;                      // per block: t offset (target-major)
    int64_t *map_v = nullptr;                     // per global V column: t index
    int *leaf_ld = nullptr;                       // per leaf: padded rows
    int64_t *leaf_lp = nullptr;                   // per leaf: prefix of padded rows (nleaf + 1)
    void *U = nullptr, *V = nullptr;
    int64_t u_elems = 0, v_elems = 0, factor_entries = 0, u_entries = 0, v_entries = 0;

    // matvec work lists and scratch
    int ngtask = 0;                               // gather tasks
    int4 *gtask = nullptr;                        // (box, row0, row1, out slot or -1)
    int64_t *gtask_pbase = nullptr;               // per task: partial base (or -1 = direct)
    int nsplit = 0;                               // boxes whose gather is split
    int *split_box = nullptr;                     // global box index
    int *split_task0 = nullptr, *split_ntask = nullptr;
    int64_t *split_pbase = nullptr;
    int64_t partial_elems = 0;
    void *t = nullptr;                            // sum_rank entries
    void *partial = nullptr;
    void *xs = nullptr;                           // N (sorted x of one column)
    // transpose product
    int64_t *tp_base = nullptr;                   // per (leaf, level<L): partial base, [(l-1)*nleaf+z]
    int64_t tpartial_elems = 0;
    void *tpartial = nullptr;
    int nsplit_T = 0;                             // boxes above the leaf level with R > 0
    int *tsplit_box = nullptr, *tsplit_level = nullptr;

    // host staging for h3d_matvec_host
    void *ey = nullptr, *eyT = nullptr;           // energy scratch: A~ q, A~^T q (N each)
    double *epart = nullptr;                      // energy partial sums
    double *fqs = nullptr, *fG = nullptr;         // forces: charges and dE/dp in Morton order
    double *fE = nullptr, *fM = nullptr;          // forces: energy partials, K(sigma,tau) scratch
    int *fctr = nullptr;                          // forces: next far-field block (work queue head)
    float4 *fph = nullptr, *fpl = nullptr;        // forces (FP32 handles): coordinates hi / lo, charge
    void *hx = nullptr, *hy = nullptr;
    int64_t host_cols = 0;

    int64_t near_interactions = 0;
    int64_t n_vertex = 0;
    double build_ms = 0;
    bool ok = false;

    size_t elem() const { return prec == H3D_FP64 ? 8 : 4; }
};

// ----------------------------------------------------------------------------
// device helpers

// FP64 kernel entry with explicitly rounded operations, used by ACA: the same
// sequence of IEEE operations as a plain C evaluation without contraction
// (d2 = fma(dz,dz,fma(dy,dy,dx*dx)), correctly rounded sqrt and division).
__device__ __forceinline__ double kernel_exact(int kind, double kappa, double ax, double ay, double az,
                                               double bx, double by, double bz) {
    double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by), dz = __dsub_rn(az, bz);
    double d2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
    if (d2 == 0.0) return 0.0;
    double r = __dsqrt_rn(d2);
    switch (kind) {
    case H3D_LAPLACE: return __ddiv_rn(H3D_INV4PI, r);
    case H3D_YUKAWA: return __ddiv_rn(__dmul_rn(H3D_INV4PI, exp(__dmul_rn(-kappa, r))), r);
    case H3D_INV_R4: return __ddiv_rn(1.0, __dmul_rn(d2, d2));
    default: return __ddiv_rn(cos(r), r);
    }
}

// Fast FP64 kernel from a squared distance (near field of FP64 products).
__device__ __forceinline__ double kernel_fast(int kind, double kappa, double d2) {
    if (d2 == 0.0) return 0.0;
    double ir = rsqrt(d2);
    switch (kind) {
    case H3D_LAPLACE: return H3D_INV4PI * ir;
    case H3D_YUKAWA: return H3D_INV4PI * exp(-kappa * d2 * ir) * ir;
    case H3D_INV_R4: return (ir * ir) * (ir * ir);
    default: return cos(d2 * ir) * ir;
    }
}

// Fast FP32 kernel from a squared distance (near field of FP32 products).
__device__ __forceinline__ float kernel_fast(int kind, float kappa, float d2) {
    if (d2 == 0.0f) return 0.0f;
    float ir = rsqrtf(d2);
    switch (kind) {
    case H3D_LAPLACE: return (float)H3D_INV4PI * ir;
    case H3D_YUKAWA: return (float)H3D_INV4PI * expf(-kappa * d2 * ir) * ir;
    case H3D_INV_R4: return (ir * ir) * (ir * ir);
    default: return cosf(d2 * ir) * ir;
    }
}

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Coordinates of a box from its Morton prefix at `level` (x bit most significant).
__host__ __device__ inline void box_coords(uint64_t key, int level, int &x, int &y, int &z) {
    x = y = z = 0;
    for (int b = 0; b < level; ++b) {
        unsigned t = (unsigned)((key >> (3 * b)) & 7ull);
        x |= ((t >> 2) & 1u) << b;
        y |= ((t >> 1) & 1u) << b;
        z |= (t & 1u) << b;
    }
}

__host__ __device__ inline uint64_t box_key_of(int x, int y, int z, int level) {
    uint64_t k = 0;
    for (int b = 0; b < level; ++b)
        k |= ((uint64_t)(((x >> b) & 1) << 2 | ((y >> b) & 1) << 1 | ((z >> b) & 1))) << (3 * b);
    return k;
}

// ----------------------------------------------------------------------------
// host-side building blocks (h3d_util.cu)
int64_t scan_exclusive(const int *in, int64_t *out, int64_t n, cudaStream_t s, Arena &tmp);
int64_t scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s, Arena &tmp);
void radix_sort_pairs(uint64_t *keys, int *vals, int64_t n, int key_bits, cudaStream_t s, Arena &tmp);
template <class T>
T read_scalar(const T *d, cudaStream_t s) {
    T v;
    H3D_CUDA(cudaMemcpyAsync(&v, d, sizeof(T), cudaMemcpyDeviceToHost, s));
    H3D_CUDA(cudaStreamSynchronize(s));
    return v;
}
int num_sms();

// Pivots given by the caller instead of searched (h3d_import_pivots): host
// arrays in the format of h3d_export_pivots.
struct FrozenPivots {
    const int *rank, *sigma, *tau;
};

// build stages
void build_tree(Handle &h, const double *points, cudaStream_t s, Arena &tmp);   // h3d_tree.cu
void build_lists(Handle &h, cudaStream_t s, Arena &tmp);                         // h3d_tree.cu
// ACA of every admissible block (pass 1: pivot search, skipped when fp is
// given) and the factors formed from the frozen pivots (pass 2)   h3d_aca.cu
void build_factors(Handle &h, cudaStream_t s, Arena &tmp, int64_t budget, const FrozenPivots *fp = nullptr);
// New coordinates for the same points (tree, lists and pivots kept): false if
// they equal the current ones bit for bit; H3D_ERR_DOMAIN for a non-finite one
bool update_points(Handle &h, const double *points, cudaStream_t s, Arena &tmp);   // h3d_tree.cu
// pass 2 again into the handle's U and V (their layout is kept)       h3d_aca.cu
void reform_factors(Handle &h, cudaStream_t s, Arena &tmp);
void refactor_skeleton(Handle &h, cudaStream_t s);                                // h3d_matvec.cu
// the points in the caller's order (device, N x 3) from the sorted copy   h3d_tree.cu
void unsorted_points(const Handle &h, double *out, cudaStream_t s);
void build_matvec_plan(Handle &h, cudaStream_t s, Arena &tmp);                   // h3d_matvec.cu
int matvec_passes(const Handle &h, int nrhs, bool transpose);  // kernel sequences one product launches
void energy(Handle &h, const void *q, double *E, void *grad, cudaStream_t s);
void forces(Handle &h, const void *q, double *E, double *F, cudaStream_t s);
void build_skeleton(Handle &h, cudaStream_t s, Arena &tmp);
void matvec_skeleton(Handle &h, const void *x, void *y, int nrhs, bool transpose, cudaStream_t s);
void run_matvec(Handle &h, const void *x, void *y, int nrhs, bool transpose, cudaStream_t s,
                cudaEvent_t *ev = nullptr);  // h3d_matvec.cu; ev: 5 events per rhs
// Symmetric storage (h3d_sym.cu): every fused pair's contribution to both of its
// boxes into the handle's FP64 accumulator (N x nq, point-major, Morton order,
// zeroed first), on the handle's sym_stream after the work already on s (ev, if
// given, is recorded when the kernel is done); then, on s after it, out (N x nq,
// point-major: the near-field buffer) += the accumulator.  nq is 1 or 8.
void sym_prepare();   // kernel attributes (once)
void sym_product(Handle &h, const void *xs, int nq, cudaStream_t s, cudaEvent_t ev = nullptr);
void sym_finish(Handle &h, void *out, int nq, cudaStream_t s);

// One persistent launch for the single-column products of many operators
// (h3d_batch.cu).  batch_plan_create returns nullptr when the handles cannot
// share one launch (skeleton storage, or FP32 and FP64 handles mixed).  The
// group sizes are the leaves per near-field item and per leaf item; lag 0
// orders the queue phase-major, lag d > 0 pipelines it over operators with a
// delay of d operators between an operator's streams and its leaves.
struct BatchPlan;
BatchPlan *batch_plan_create(const std::vector<Handle *> &hs, int near_group, int leaf_group, int lag);
void batch_plan_regroup(BatchPlan &p, int near_group, int leaf_group, int lag);
// leaves per near-field item and per leaf item chosen per operator
void batch_plan_set_groups(BatchPlan &p, const int *near_groups, const int *leaf_groups, int lag);
void batch_plan_op_groups(const BatchPlan &p, int *near_groups, int *leaf_groups);
void batch_plan_groups(const BatchPlan &p, int *near_group, int *leaf_group, int *lag);
int batch_plan_max_ctas_per_sm(const BatchPlan &p);
void batch_plan_run(BatchPlan &p, const void *const *x, void *const *y, int ctas_per_sm, cudaStream_t s);
// the caller's queue (false if an item is out of range; NULL items: the queue
// of the current settings again), the queue in use, the bound of every wait
bool batch_plan_set_queue(BatchPlan &p, const int *items, int64_t count);
void batch_plan_get_queue(const BatchPlan &p, int *items, int64_t cap, int64_t *count);
void batch_plan_set_wait(BatchPlan &p, long long ns);
void batch_plan_free(BatchPlan *p);

}  // namespace h3d
