// h3d_batch.cu -- the single-column products y_i = A~_i x_i of many operators
// (independent point clouds, each with its own tree, kernel and factors) in ONE
// persistent launch (Alg. 2 for every operator at once), captured with the
// reset of its queue into a CUDA graph.
//
// The work items of all operators sit in one device queue (P first, then the
// rest phase-major or pipelined over operators; see build_items):
//   P  permute a chunk of points: xs = x[perm]                         (A5)
//   G  one gather task: t_b = V_b^T xs(Y_b) over a row range           (A7)
//   N  near field of a run of leaves (one leaf per warp) into the near
//      buffer                                                         (A6)
//   R  sum of the row-range partials of one split source box           (A7)
//   L  a run of leaves: y(Z) = sum over levels of U panel * t, plus the
//      near sum, written in the caller's order                         (A8, A9)
// The G and N items of an operator are interleaved, so the CTAs that share an
// SM mix HBM-bound factor streams with ALU-bound near-field tiles; the kernel
// is held to 72 registers and a three-buffer leaf ring so that seven CTAs fit
// on an SM (at 64 registers, eight would fit, but the spills cost more than
// the extra CTA gains).  A CTA takes its next item with one atomic on the queue head
// (fetched while the current item runs).  An item whose inputs are incomplete
// waits on its operator's completion counters: G and N wait for every P of the
// operator, R for every G, L for every G, R and N.  Items wait only on items
// that sit earlier in the queue and so were taken by CTAs that are already
// running; every wait therefore ends.  Each is still bounded (by a limit in
// nanoseconds of the GPU's global timer, 2 s unless the caller sets another):
// a CTA that gives up records H3D_ERR_TIMEOUT in the operator's error word,
// raises the batch's abort flag (on which the other CTAs stop) and leaves.
//
// Visibility: a finished item's CTA synchronises, then one thread fences at GPU
// scope and adds 1 to the counter; a waiting thread reads the counter with an
// acquire load, and its CTA synchronises before use.  Values written inside the
// launch (xs, t, partials, near sums) are never read through the read-only path:
// through L2 only where they are read once, through L1 (ld.global.ca) where
// neighbouring leaves read them again (after the acquire).
#include <algorithm>
#include <type_traits>
#include <vector>

#include "h3d_async.cuh"
#include "h3d_internal.cuh"
#include "h3d_stream.cuh"

namespace h3d {

namespace {

constexpr int kBatchThreads = kLeafThreads;
constexpr int kPermChunk = 1024;                       // points per P item
constexpr int kPermPerThread = kPermChunk / kBatchThreads;
constexpr int kBatchCtasPerSm = 7;   // resident CTAs the register budget is set for (72 registers)
// k_batch's leaf ring: one buffer fewer than k_leaf's (shared memory for seven or eight CTAs per SM)
constexpr int kBatchStages = kStages - 1;
// dynamic shared memory, one region per item kind (they overlap):
//   L  ring of kBatchStages * kChunkBytes, then the leaf reduction buffer
//   G  source values (kTaskMaxRows) at 0, reduction buffer at kRedOff
//   N  per warp: kNearWarpSrc staged sources (32 B each) from 0, then the
//      near-list prefixes (kNearWarpLists + 1 ints per warp) at kNearPreOff
constexpr size_t kRedOff = 16384;
constexpr size_t kNearPreOff = (size_t)(kBatchThreads / 32) * kNearWarpSrc * 32;
constexpr size_t kLeafRedOff = (size_t)kBatchStages * kChunkBytes;
constexpr size_t kBatchDynSmem = kLeafRedOff + kLeafThreads * 16;

static_assert(kTaskMaxRows * sizeof(double) <= kRedOff, "gather rows overlap the reduction buffer");
static_assert(kRedOff + kLeafThreads * 16 <= kBatchDynSmem, "gather reduction buffer out of range");
static_assert(kNearPreOff + (kBatchThreads / 32) * (kNearWarpLists + 1) * sizeof(int) <= kBatchDynSmem,
              "near staging out of range");
static_assert(kPermChunk % kBatchThreads == 0, "P items split evenly over the threads");

enum : int { kItemGather = 0, kItemNear = 1, kItemReduce = 2, kItemLeaf = 3, kItemPerm = 4 };

struct BatchOp {
    GatherArgs G;
    SplitArgs S;
    LeafArgs A;
    const void *V, *U;
    void *xs, *t, *partial, *nearbuf;
    const int *perm;
    int64_t N;
    int ngtask, nsplit, nnear, nperm;   // items of the G, R, N and P phases
};

struct BatchArgs {
    const BatchOp *ops;
    const int4 *items;         // (operator, kind, first, count)
    int nitems;
    int *head;                 // next free queue slot
    int *abort;
    int4 *done;                // per operator: finished (G, R, N, P) items
    const void *const *xy;     // per operator: x, y (device pointers)
    long long wait_ns;         // bound of every wait on a completion counter
};

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

// true once *cnt >= target; false on abort or after wait_ns nanoseconds
__device__ bool wait_count(const int *cnt, int target, const int *abort, long long wait_ns) {
    if (ld_acquire(cnt) >= target) return true;
    const long long t0 = global_ns();
    while (ld_acquire(cnt) < target) {
        if (ld_acquire(abort)) return false;
        if (global_ns() - t0 > wait_ns) return false;
        __nanosleep(128);
    }
    return true;
}

// the operator's arguments into shared memory, by the whole CTA
__device__ __forceinline__ void load_op(const BatchOp *src_op, BatchOp &O) {
    const int *src = reinterpret_cast<const int *>(src_op);
    int *dst = reinterpret_cast<int *>(&O);
    for (int k = threadIdx.x; k < (int)(sizeof(BatchOp) / sizeof(int)); k += blockDim.x) dst[k] = __ldg(src + k);
}

template <class T>
__global__ void __launch_bounds__(kBatchThreads, kBatchCtasPerSm) k_batch(BatchArgs B) {
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ __align__(8) uint64_t bars[kBatchStages];
    __shared__ ChunkPlan P;
    __shared__ int s_next[2], s_ok;
    __shared__ __align__(16) BatchOp O;   // the current item's operator
    if (threadIdx.x == 0) {
        for (int q = 0; q < kBatchStages; ++q) mbar_init(&bars[q], 1);
        mbar_fence_init();
        s_next[0] = atomicAdd(B.head, 1);
    }
    __syncthreads();
    uint32_t ring = 0;   // chunks taken through the leaf ring so far
    for (int iter = 0;; ++iter) {
        const int it = s_next[iter & 1];
        if (it >= B.nitems) break;
        const int4 I = B.items[it];
        int4 *done = B.done + I.x;
        load_op(B.ops + I.x, O);   // the previous item is finished with O
        if (threadIdx.x == 0) {
            s_next[(iter + 1) & 1] = atomicAdd(B.head, 1);
            bool ok = true;
            const BatchOp &G = B.ops[I.x];
            const long long lim = B.wait_ns;
            if (I.y == kItemGather || I.y == kItemNear) ok = wait_count(&done->w, G.nperm, B.abort, lim);
            else if (I.y == kItemReduce) ok = wait_count(&done->x, G.ngtask, B.abort, lim);
            else if (I.y == kItemLeaf)
                ok = wait_count(&done->x, G.ngtask, B.abort, lim) && wait_count(&done->y, G.nsplit, B.abort, lim) &&
                     wait_count(&done->z, G.nnear, B.abort, lim);
            if (!ok) {
                if (!ld_acquire(B.abort)) atomicCAS(G.A.err, 0, (int)H3D_ERR_TIMEOUT);
                atomicExch(B.abort, 1);
            }
            __threadfence();
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
        if (I.y == kItemPerm) {   // all loads of a thread in flight together
            const T *x = static_cast<const T *>(B.xy[2 * I.x]);
            T *xs = static_cast<T *>(O.xs);
            int idx[kPermPerThread];
            T v[kPermPerThread];
#pragma unroll
            for (int k = 0; k < kPermPerThread; ++k) {
                const int64_t i = (int64_t)I.z + threadIdx.x + k * kBatchThreads;
                idx[k] = i < O.N ? O.perm[i] : -1;
            }
#pragma unroll
            for (int k = 0; k < kPermPerThread; ++k) v[k] = idx[k] >= 0 ? x[idx[k]] : T(0);
#pragma unroll
            for (int k = 0; k < kPermPerThread; ++k)
                if (idx[k] >= 0) xs[I.z + threadIdx.x + k * kBatchThreads] = v[k];
        } else if (I.y == kItemGather) {
            gather_task<T, kBatchThreads, 8, true>(O.G, I.z, static_cast<const T *>(O.V), static_cast<const T *>(O.xs),
                                                   static_cast<T *>(O.t), static_cast<T *>(O.partial),
                                                   reinterpret_cast<T *>(dyn), reinterpret_cast<T *>(dyn + kRedOff));
        } else if (I.y == kItemNear) {   // one leaf per warp at a time
            const int w = threadIdx.x >> 5;
            using Src = typename std::conditional<sizeof(T) == 4, float4, Pt4d>::type;
            Src *wsrc = reinterpret_cast<Src *>(dyn) + w * (sizeof(T) == 4 ? 2 : 1) * kNearWarpSrc;
            int *wpre = reinterpret_cast<int *>(dyn + kNearPreOff) + w * (kNearWarpLists + 1);
            for (int z = I.z + w; z < I.z + I.w; z += kBatchThreads / 32)
                near_warp(O.A, z, static_cast<const T *>(O.xs), static_cast<T *>(O.nearbuf), wsrc, wpre);
        } else if (I.y == kItemReduce) {
            reduce_split<T, true>(O.S, I.z, kBatchThreads, static_cast<const T *>(O.partial), static_cast<T *>(O.t));
        } else {
            T *y = static_cast<T *>(const_cast<void *>(B.xy[2 * I.x + 1]));
            bool ok = true;
            for (int z = I.z; z < I.z + I.w && ok; ++z) {
                ok = leaf_task<T, true, kBatchStages>(O.A, z, static_cast<const T *>(O.U), static_cast<const T *>(O.t),
                                                      static_cast<const T *>(O.nearbuf), y, dyn, bars, P,
                                                      reinterpret_cast<T *>(dyn + kLeafRedOff), ring);
                __syncthreads();
            }
            if (!ok) {
                if (threadIdx.x == 0) atomicExch(B.abort, 1);
                break;
            }
        }
        // the next item may hand this shared memory to bulk copies (async proxy)
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0 && I.y != kItemLeaf) {
            __threadfence();
            atomicAdd(I.y == kItemGather ? &done->x : I.y == kItemReduce ? &done->y : I.y == kItemNear ? &done->z
                                                                                                     : &done->w, 1);
        }
    }
}

}  // namespace

struct BatchPlan {
    int elem = 4;                            // 4: FP32 operators, 8: FP64
    int nops = 0;
    int near_group = 0, leaf_group = 0, lag = 0;   // the last groups set for every operator
    std::vector<int> ng, lg;                 // per operator: leaves per near-field item and per leaf item
    std::vector<BatchOp> ops;
    std::vector<Handle *> hs;
    Arena mem;
    void *d_ops = nullptr, *d_items = nullptr, *d_xy = nullptr;
    int *d_state = nullptr;                  // head, abort, pad, pad, then done[nops] (int4 each)
    int nitems = 0;
    std::vector<int4> items;                 // the queue on the device
    bool custom = false;                     // queue given by the caller (batch_plan_set_queue)
    long long wait_ns = 2000000000LL;        // bound of every wait (2 s)
    std::vector<const void *> xy;            // the pointers last copied to d_xy
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    int exec_ctas = 0;
    ~BatchPlan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (cap) cudaStreamDestroy(cap);
    }
};

namespace {

template <class V>
void *upload(BatchPlan &p, void *old, const std::vector<V> &v) {
    if (old) p.mem.free_one(old);
    void *d = p.mem.alloc(std::max<size_t>(1, v.size()) * sizeof(V));
    if (!v.empty()) H3D_CUDA(cudaMemcpy(d, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice));
    return d;
}

// Merge two item lists, keeping each list's order and spreading b evenly
// among a.
void merge_even(std::vector<int4> &out, const std::vector<int4> &a, const std::vector<int4> &b) {
    size_t ia = 0, ib = 0;
    while (ia < a.size() || ib < b.size()) {
        if (ib < b.size() && (ia >= a.size() || (int64_t)ib * (int64_t)a.size() <= (int64_t)ia * (int64_t)b.size()))
            out.push_back(b[ib++]);
        else
            out.push_back(a[ia++]);
    }
}

// The queue: P of every operator first.  Then, with lag 0, phase-major: the G
// and N items of every operator (an operator's near runs spread evenly among
// its gather tasks), then every R, then every L.  With lag d > 0, pipelined
// over operators: round k holds the G and N items of operator k merged with
// the R and L items of operator k - d, so that operators finish one after
// another instead of all at the end.  Either way every item comes after the
// items it waits for.
struct QueueCounts {
    int64_t n;             // points
    int ngtask, nsplit, nleaf;
};

std::vector<int4> batch_queue(const std::vector<QueueCounts> &c, const std::vector<int> &ng,
                              const std::vector<int> &lg, int lag) {
    const int nops = (int)c.size();
    std::vector<int4> items;
    for (int o = 0; o < nops; ++o)
        for (int64_t i = 0; i < c[o].n; i += kPermChunk) items.push_back(make_int4(o, kItemPerm, (int)i, 0));
    auto stream_items = [&](int o) {   // G and N of operator o
        std::vector<int4> g, n, out;
        for (int k = 0; k < c[o].ngtask; ++k) g.push_back(make_int4(o, kItemGather, k, 1));
        for (int z0 = 0; z0 < c[o].nleaf; z0 += ng[o])
            n.push_back(make_int4(o, kItemNear, z0, std::min(ng[o], c[o].nleaf - z0)));
        merge_even(out, g, n);
        return out;
    };
    auto finish_items = [&](int o, bool reduce, bool leaf) {   // R and / or L of operator o
        std::vector<int4> out;
        if (reduce)
            for (int q = 0; q < c[o].nsplit; ++q) out.push_back(make_int4(o, kItemReduce, q, 1));
        if (leaf)
            for (int z0 = 0; z0 < c[o].nleaf; z0 += lg[o])
                out.push_back(make_int4(o, kItemLeaf, z0, std::min(lg[o], c[o].nleaf - z0)));
        return out;
    };
    if (lag <= 0) {
        for (int o = 0; o < nops; ++o) {
            const std::vector<int4> v = stream_items(o);
            items.insert(items.end(), v.begin(), v.end());
        }
        for (int o = 0; o < nops; ++o) {
            const std::vector<int4> v = finish_items(o, true, false);
            items.insert(items.end(), v.begin(), v.end());
        }
        for (int o = 0; o < nops; ++o) {
            const std::vector<int4> v = finish_items(o, false, true);
            items.insert(items.end(), v.begin(), v.end());
        }
    } else {
        for (int k = 0; k < nops + lag; ++k) {
            const std::vector<int4> a = k < nops ? stream_items(k) : std::vector<int4>();
            const std::vector<int4> b = k >= lag ? finish_items(k - lag, true, true) : std::vector<int4>();
            merge_even(items, a, b);
        }
    }
    return items;
}

void drop_graph(BatchPlan &p) {
    if (p.exec) {
        H3D_CUDA(cudaGraphExecDestroy(p.exec));
        p.exec = nullptr;
    }
}

void set_items(BatchPlan &p, const std::vector<int4> &items) {
    p.items = items;
    p.nitems = (int)items.size();
    p.d_items = upload(p, p.d_items, items);
    drop_graph(p);
}

void build_items(BatchPlan &p) {
    std::vector<QueueCounts> c;
    for (const Handle *h : p.hs) c.push_back(QueueCounts{h->N, h->ngtask, h->nsplit, h->nleaf});
    set_items(p, batch_queue(c, p.ng, p.lg, p.lag));
    p.custom = false;
}

}  // namespace

BatchPlan *batch_plan_create(const std::vector<Handle *> &hs, int near_group, int leaf_group, int lag) {
    if (hs.empty()) return nullptr;
    const int elem = hs[0]->prec == H3D_FP64 ? 8 : 4;
    for (Handle *h : hs)
        if (h->storage != H3D_STORE_FACTORS || (h->prec == H3D_FP64 ? 8 : 4) != elem) return nullptr;
    BatchPlan *p = new BatchPlan;
    try {
        p->elem = elem;
        p->hs = hs;
        p->nops = (int)hs.size();
        for (int o = 0; o < p->nops; ++o) {
            const Handle &h = *hs[o];
            BatchOp op{};
            op.G = GatherArgs{h.gtask, h.gtask_pbase, h.box_start, h.Rv, h.ldv, h.vbase, h.vcol0, h.map_v};
            op.S = SplitArgs{h.split_box, h.split_ntask, h.split_pbase, h.Rv, h.ldv, h.vcol0, h.map_v};
            op.A = leaf_args(h);
            op.V = h.V;
            op.U = h.U;
            op.xs = h.xs;
            op.N = h.N;
            op.nperm = (int)((h.N + kPermChunk - 1) / kPermChunk);
            op.t = h.t;
            op.partial = h.partial;
            op.nearbuf = h.nearbuf;
            op.perm = h.perm;
            op.ngtask = h.ngtask;
            op.nsplit = h.nsplit;
            p->ops.push_back(op);
        }
        batch_plan_regroup(*p, near_group, leaf_group, lag);
        p->d_state = p->mem.get<int>((size_t)(p->nops + 1) * 4);
        p->d_xy = p->mem.alloc((size_t)p->nops * 2 * sizeof(void *));
        H3D_CUDA(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
    } catch (...) {
        delete p;
        throw;
    }
    return p;
}

void batch_plan_regroup(BatchPlan &p, int near_group, int leaf_group, int lag) {
    p.near_group = std::max(1, near_group);
    p.leaf_group = std::max(1, leaf_group);
    p.ng.assign(p.nops, p.near_group);
    p.lg.assign(p.nops, p.leaf_group);
    batch_plan_set_groups(p, p.ng.data(), p.lg.data(), lag);
}

void batch_plan_set_groups(BatchPlan &p, const int *near_groups, const int *leaf_groups, int lag) {
    p.lag = std::max(0, lag);
    p.ng.resize(p.nops);
    p.lg.resize(p.nops);
    for (int o = 0; o < p.nops; ++o) {
        p.ng[o] = std::max(1, near_groups[o]);
        p.lg[o] = std::max(1, leaf_groups[o]);
        p.ops[o].nnear = (p.hs[o]->nleaf + p.ng[o] - 1) / p.ng[o];
    }
    p.d_ops = upload(p, p.d_ops, p.ops);
    build_items(p);
}

void batch_plan_op_groups(const BatchPlan &p, int *near_groups, int *leaf_groups) {
    for (int o = 0; o < p.nops; ++o) {
        if (near_groups) near_groups[o] = p.ng[o];
        if (leaf_groups) leaf_groups[o] = p.lg[o];
    }
}

bool batch_plan_set_queue(BatchPlan &p, const int *items, int64_t count) {
    if (!items) {   // back to the queue of the current settings
        build_items(p);
        return true;
    }
    std::vector<int4> q;
    for (int64_t k = 0; k < count; ++k) {
        const int4 it = make_int4(items[4 * k], items[4 * k + 1], items[4 * k + 2], items[4 * k + 3]);
        if (it.x < 0 || it.x >= p.nops) return false;
        const Handle &h = *p.hs[it.x];
        bool ok = false;
        switch (it.y) {
        case kItemGather: ok = it.z >= 0 && it.z < h.ngtask; break;
        case kItemReduce: ok = it.z >= 0 && it.z < h.nsplit; break;
        case kItemNear:
        case kItemLeaf: ok = it.z >= 0 && it.w >= 1 && (int64_t)it.z + it.w <= h.nleaf; break;
        case kItemPerm: ok = it.z >= 0 && it.z < h.N; break;
        default: ok = false;
        }
        if (!ok) return false;
        q.push_back(it);
    }
    set_items(p, q);
    p.custom = true;
    return true;
}

void batch_plan_get_queue(const BatchPlan &p, int *items, int64_t cap, int64_t *count) {
    *count = (int64_t)p.items.size();
    if (!items) return;
    for (int64_t k = 0; k < std::min<int64_t>(cap, (int64_t)p.items.size()); ++k) {
        items[4 * k] = p.items[k].x;
        items[4 * k + 1] = p.items[k].y;
        items[4 * k + 2] = p.items[k].z;
        items[4 * k + 3] = p.items[k].w;
    }
}

void batch_plan_set_wait(BatchPlan &p, long long ns) {
    p.wait_ns = ns;
    drop_graph(p);
}

void batch_plan_groups(const BatchPlan &p, int *near_group, int *leaf_group, int *lag) {
    *near_group = p.near_group;
    *leaf_group = p.leaf_group;
    *lag = p.lag;
}

int batch_plan_max_ctas_per_sm(const BatchPlan &p) {
    int n = 0;
    if (p.elem == 8) H3D_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<double>, kBatchThreads, kBatchDynSmem));
    else H3D_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<float>, kBatchThreads, kBatchDynSmem));
    return std::max(1, n);
}

void batch_plan_run(BatchPlan &p, const void *const *x, void *const *y, int ctas_per_sm, cudaStream_t s) {
    ctas_per_sm = std::max(1, std::min(ctas_per_sm, batch_plan_max_ctas_per_sm(p)));
    bool same = (int)p.xy.size() == 2 * p.nops;
    for (int o = 0; o < p.nops && same; ++o) same = p.xy[2 * o] == x[o] && p.xy[2 * o + 1] == y[o];
    if (!same) {
        p.xy.resize(2 * p.nops);
        for (int o = 0; o < p.nops; ++o) {
            p.xy[2 * o] = x[o];
            p.xy[2 * o + 1] = y[o];
        }
        // pageable source: the copy has taken the values when the call returns
        H3D_CUDA(cudaMemcpyAsync(p.d_xy, p.xy.data(), p.xy.size() * sizeof(void *), cudaMemcpyHostToDevice, s));
    }
    if (!p.exec || p.exec_ctas != ctas_per_sm) {
        if (p.exec) {
            H3D_CUDA(cudaGraphExecDestroy(p.exec));
            p.exec = nullptr;
        }
        int *st = p.d_state;
        BatchArgs a{static_cast<const BatchOp *>(p.d_ops), static_cast<const int4 *>(p.d_items), p.nitems, st, st + 1,
                    reinterpret_cast<int4 *>(st + 4), static_cast<const void *const *>(p.d_xy), p.wait_ns};
        const int grid = std::max(1, std::min(p.nitems, ctas_per_sm * num_sms()));
        cudaGraph_t g = nullptr;
        H3D_CUDA(cudaStreamBeginCapture(p.cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t le = cudaMemsetAsync(st, 0, (size_t)(p.nops + 1) * sizeof(int4), p.cap);
        if (le == cudaSuccess) {
            if (p.elem == 8) k_batch<double><<<grid, kBatchThreads, kBatchDynSmem, p.cap>>>(a);
            else k_batch<float><<<grid, kBatchThreads, kBatchDynSmem, p.cap>>>(a);
            le = cudaGetLastError();
        }
        const cudaError_t ce = cudaStreamEndCapture(p.cap, &g);
        if (le == cudaSuccess) le = ce;
        if (le != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            H3D_CUDA(le);
        }
        const cudaError_t e = cudaGraphInstantiate(&p.exec, g, 0);
        cudaGraphDestroy(g);
        H3D_CUDA(e);
        p.exec_ctas = ctas_per_sm;
    }
    H3D_CUDA(cudaGraphLaunch(p.exec, s));
}

void batch_plan_free(BatchPlan *p) { delete p; }

}  // namespace h3d

extern "C" h3d_status h3d_batch_queue(int nops, const int64_t *n_points, const int *n_gather, const int *n_split,
                                      const int *n_leaves, int near_group, int leaf_group, int lag, int *items,
                                      int64_t cap, int64_t *count) {
    if (nops < 1 || !n_points || !n_gather || !n_split || !n_leaves || near_group < 1 || leaf_group < 1 || lag < 0 ||
        !count || cap < 0)
        return H3D_ERR_ARG;
    std::vector<h3d::QueueCounts> c;
    for (int o = 0; o < nops; ++o) {
        if (n_points[o] < 1 || n_gather[o] < 0 || n_split[o] < 0 || n_leaves[o] < 1) return H3D_ERR_ARG;
        c.push_back(h3d::QueueCounts{n_points[o], n_gather[o], n_split[o], n_leaves[o]});
    }
    try {
        const std::vector<int4> q = h3d::batch_queue(c, std::vector<int>(nops, near_group),
                                                     std::vector<int>(nops, leaf_group), lag);
        *count = (int64_t)q.size();
        if (!items) return H3D_OK;
        if (cap < (int64_t)q.size()) return H3D_ERR_ARG;
        for (size_t k = 0; k < q.size(); ++k) {
            items[4 * k] = q[k].x;
            items[4 * k + 1] = q[k].y;
            items[4 * k + 2] = q[k].z;
            items[4 * k + 3] = q[k].w;
        }
    } catch (const std::bad_alloc &) {
        return H3D_ERR_OOM;
    }
    return H3D_OK;
}
