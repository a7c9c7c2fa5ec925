// h3d_api.cu -- the extern "C" entry points declared in include/h3d.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "h3d_internal.cuh"

using h3d::Handle;

// The handle owns its Handle through a pointer, so that h3d_import_pivots can
// build a replacement and swap it in only once that build has succeeded.
struct h3d_handle_s {
    Handle *p = nullptr;
    ~h3d_handle_s() { delete p; }
};

namespace {

template <class F>
h3d_status guard(F &&f) {
    try {
        f();
        return H3D_OK;
    } catch (const h3d::Error &e) {
        return e.st;
    } catch (const std::bad_alloc &) {
        return H3D_ERR_OOM;
    }
}

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

void h3d_default_options(h3d_options *opt) {
    if (!opt) return;
    opt->precision = H3D_FP32_3XTF32;
    opt->kappa = 1.0;
    opt->rank_cap = h3d::kMaxRank;
    opt->lo[0] = opt->lo[1] = opt->lo[2] = -1.0;
    opt->side = 2.0;
    opt->workspace_bytes = 0;
    opt->admissibility = H3D_ADM_HODLR3D;
    opt->storage = H3D_STORE_FACTORS;
}

const char *h3d_status_string(h3d_status s) {
    switch (s) {
    case H3D_OK: return "ok";
    case H3D_ERR_ARG: return "invalid argument";
    case H3D_ERR_DOMAIN: return "point outside the domain cube (or not finite)";
    case H3D_ERR_OOM: return "device allocation failed";
    case H3D_ERR_CUDA: return "CUDA error";
    case H3D_ERR_ACA_RANK: return "ACA did not reach the tolerance within rank_cap";
    case H3D_ERR_TIMEOUT: return "bounded device wait timed out";
    case H3D_ERR_STATE: return "handle unusable";
    case H3D_ERR_DEPTH: return "tree depth would exceed 21 (too many coincident points)";
    }
    return "unknown status";
}

namespace {

// Everything the build computes, into the parameters already set in h: tree,
// lists, ACA (pivots searched, or the caller's when fp is given), factor layout
// and product plan.  Synchronises s.
h3d_status build_into(Handle &h, const double *points, cudaStream_t s, const h3d::FrozenPivots *fp) {
    const auto t0 = std::chrono::steady_clock::now();
    h3d_status st = guard([&] {
        h3d::Arena tmp;
        h.d_err = h.mem.get<int>(1);
        H3D_CUDA(cudaHostAlloc((void **)&h.h_async_err, sizeof(int), cudaHostAllocMapped));
        *h.h_async_err = 0;
        H3D_CUDA(cudaHostGetDevicePointer((void **)&h.d_async_err, h.h_async_err, 0));
        h3d::build_tree(h, points, s, tmp);
        h3d::build_lists(h, s, tmp);
        h3d::build_factors(h, s, tmp, h.budget, fp);
        h3d::build_matvec_plan(h, s, tmp);
        H3D_CUDA(cudaStreamSynchronize(s));
    });
    if (st != H3D_OK) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        return st;
    }
    h.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    h.ok = true;
    return H3D_OK;
}

// a new Handle with the parameters of h (nothing built)
Handle *same_parameters(const Handle &h) {
    Handle *n = new (std::nothrow) Handle;
    if (!n) return nullptr;
    n->N = h.N;
    n->kernel = h.kernel;
    n->prec = h.prec;
    n->tf32 = h.tf32;
    n->leaf_size = h.leaf_size;
    n->rank_cap = h.rank_cap;
    n->adm = h.adm;
    n->storage = h.storage;
    n->budget = h.budget;
    n->tol = h.tol;
    n->kappa = h.kappa;
    n->side = h.side;
    for (int d = 0; d < 3; ++d) n->lo[d] = h.lo[d];
    return n;
}

}  // namespace

h3d_status h3d_build(const double *points, int64_t N, h3d_kernel kernel, int leaf_size, double tol,
                     const h3d_options *opt, void *stream, h3d_handle *out) {
    if (!out || !points || N < 1 || N >= (int64_t)1 << 31) return H3D_ERR_ARG;
    if (leaf_size < 1 || leaf_size > h3d::kMaxLeaf || !(tol >= 0.0) || !std::isfinite(tol)) return H3D_ERR_ARG;
    if ((int)kernel < 0 || (int)kernel > 3) return H3D_ERR_ARG;
    h3d_options o;
    h3d_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != H3D_FP32 && o.precision != H3D_FP64 && o.precision != H3D_FP32_3XTF32) return H3D_ERR_ARG;
    if (o.rank_cap < 1 || o.rank_cap > h3d::kMaxRank) return H3D_ERR_ARG;
    if (!(o.side > 0.0) || !std::isfinite(o.side)) return H3D_ERR_ARG;
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(o.lo[d])) return H3D_ERR_ARG;
    if (!(o.kappa >= 0.0) || !std::isfinite(o.kappa)) return H3D_ERR_ARG;
    if (o.admissibility < H3D_ADM_HODLR3D || o.admissibility > H3D_ADM_WEAK) return H3D_ERR_ARG;
    if (o.storage != H3D_STORE_FACTORS && o.storage != H3D_STORE_SKELETON && o.storage != H3D_STORE_SYMMETRIC)
        return H3D_ERR_ARG;
    if (o.workspace_bytes < 0) return H3D_ERR_ARG;
    if (!is_device_ptr(points)) return H3D_ERR_ARG;

    h3d_handle_s *hs = new (std::nothrow) h3d_handle_s;
    if (!hs) return H3D_ERR_OOM;
    hs->p = new (std::nothrow) Handle;
    if (!hs->p) {
        delete hs;
        return H3D_ERR_OOM;
    }
    Handle &h = *hs->p;
    h.N = N;
    h.kernel = kernel;
    h.prec = o.precision == H3D_FP64 ? H3D_FP64 : H3D_FP32;
    h.tf32 = o.precision == H3D_FP32_3XTF32;
    h.leaf_size = leaf_size;
    h.rank_cap = o.rank_cap;
    h.adm = o.admissibility;
    h.storage = o.storage;
    h.budget = o.workspace_bytes;
    h.tol = tol;
    h.kappa = o.kappa;
    h.side = o.side;
    for (int d = 0; d < 3; ++d) h.lo[d] = o.lo[d];
    const h3d_status st = build_into(h, points, as_stream(stream), nullptr);
    if (st != H3D_OK) {
        delete hs;
        return st;
    }
    *out = hs;
    return H3D_OK;
}

// The status a product kernel left in the handle's error word (a bounded wait
// that gave up), reported once: reading it clears it.
static h3d_status async_error(const Handle &h) {
    if (*(volatile int *)h.h_async_err == 0) return H3D_OK;
    const int e = __atomic_exchange_n(h.h_async_err, 0, __ATOMIC_SEQ_CST);
    return e ? (h3d_status)e : H3D_OK;
}

static h3d_status matvec_common(h3d_handle hh, const void *x, void *y, int nrhs, void *stream, bool transpose) {
    if (!hh) return H3D_ERR_ARG;
    Handle &h = *hh->p;
    if (!h.ok) return H3D_ERR_STATE;
    if (h3d_status e = async_error(h)) return e;
    if (!x || !y || nrhs < 1 || x == y) return H3D_ERR_ARG;
    return guard([&] { h3d::run_matvec(h, x, y, nrhs, transpose, as_stream(stream)); });
}

h3d_status h3d_matvec(h3d_handle h, const void *x, void *y, int nrhs, void *stream) {
    return matvec_common(h, x, y, nrhs, stream, false);
}

h3d_status h3d_matvec_T(h3d_handle h, const void *x, void *y, int nrhs, void *stream) {
    return matvec_common(h, x, y, nrhs, stream, true);
}

h3d_status h3d_energy(h3d_handle hh, const void *q, double *E, void *grad, void *stream) {
    if (!hh) return H3D_ERR_ARG;
    Handle &h = *hh->p;
    if (!h.ok) return H3D_ERR_STATE;
    if (h3d_status e = async_error(h)) return e;
    if (!q || !E || q == grad) return H3D_ERR_ARG;
    return guard([&] { h3d::energy(h, q, E, grad, as_stream(stream)); });
}

h3d_status h3d_forces(h3d_handle hh, const void *q, double *E, double *F, void *stream) {
    if (!hh) return H3D_ERR_ARG;
    Handle &h = *hh->p;
    if (!h.ok) return H3D_ERR_STATE;
    if (h3d_status e = async_error(h)) return e;
    if (!q || !E || !F) return H3D_ERR_ARG;
    return guard([&] { h3d::forces(h, q, E, F, as_stream(stream)); });
}

h3d_status h3d_matvec_host(h3d_handle hh, const void *x_host, void *y_host, int nrhs, void *stream) {
    if (!hh) return H3D_ERR_ARG;
    Handle &h = *hh->p;
    if (!h.ok) return H3D_ERR_STATE;
    if (h3d_status e = async_error(h)) return e;
    if (!x_host || !y_host || nrhs < 1) return H3D_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    return guard([&] {
        const size_t bytes = (size_t)h.N * (size_t)nrhs * h.elem();
        if (h.host_cols < nrhs) {
            H3D_CUDA(cudaStreamSynchronize(s));
            if (h.hx) h.mem.free_one(h.hx);
            if (h.hy) h.mem.free_one(h.hy);
            h.hx = h.hy = nullptr;
            h.host_cols = 0;
            h.hx = h.mem.alloc(bytes);
            h.hy = h.mem.alloc(bytes);
            h.host_cols = nrhs;
        }
        H3D_CUDA(cudaMemcpyAsync(h.hx, x_host, bytes, cudaMemcpyHostToDevice, s));
        h3d::run_matvec(h, h.hx, h.hy, nrhs, false, s);
        H3D_CUDA(cudaMemcpyAsync(y_host, h.hy, bytes, cudaMemcpyDeviceToHost, s));
        H3D_CUDA(cudaStreamSynchronize(s));
    });
}

h3d_status h3d_matvec_profile(h3d_handle hh, const void *x, void *y, int nrhs, void *stream, float *phase_ms,
                              int nphase) {
    if (!hh || !phase_ms || nphase < 1) return H3D_ERR_ARG;
    Handle &h = *hh->p;
    if (!h.ok) return H3D_ERR_STATE;
    if (h.storage == H3D_STORE_SKELETON) return H3D_ERR_ARG;   // phases of the factor-streaming product only
    if (!x || !y || nrhs < 1 || x == y) return H3D_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    std::vector<cudaEvent_t> ev((size_t)5 * nrhs, nullptr);
    h3d_status st = guard([&] {
        for (auto &e : ev) H3D_CUDA(cudaEventCreate(&e));
        h3d::run_matvec(h, x, y, nrhs, false, s, ev.data());
        H3D_CUDA(cudaStreamSynchronize(s));
        float acc[4] = {0, 0, 0, 0};
        const int passes = h3d::matvec_passes(h, nrhs, false);
        for (int c = 0; c < passes; ++c)
            for (int p = 0; p < 4; ++p) {
                float ms = 0;
                H3D_CUDA(cudaEventElapsedTime(&ms, ev[5 * c + p], ev[5 * c + p + 1]));
                acc[p] += ms;
            }
        for (int p = 0; p < nphase && p < 4; ++p) phase_ms[p] = acc[p];
    });
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    return st;
}

void h3d_debug_fail_alloc(int64_t after) { h3d::fail_alloc_countdown() = after < 0 ? -1 : after; }

h3d_status h3d_free(h3d_handle hh) {
    if (!hh) return H3D_OK;
    cudaDeviceSynchronize();
    delete hh;
    return H3D_OK;
}

h3d_status h3d_get_stats(h3d_handle hh, h3d_stats *st) {
    if (!hh || !st) return H3D_ERR_ARG;
    const Handle &h = *hh->p;
    if (!h.ok) return H3D_ERR_STATE;
    std::memset(st, 0, sizeof(*st));
    st->N = h.N;
    st->depth = h.L;
    st->precision = h.tf32 ? H3D_FP32_3XTF32 : h.prec;
    st->kernel = h.kernel;
    st->leaf_size = h.leaf_size;
    st->tol = h.tol;
    st->n_boxes = h.n_boxes;
    st->n_leaves = h.nleaf;
    st->n_blocks = h.nblk;
    st->n_near = h.nnear;
    st->max_rank = h.max_rank;
    st->sum_rank = h.sum_rank;
    st->factor_entries = h.factor_entries;
    st->u_entries = h.u_entries;
    st->v_entries = h.v_entries;
    st->factor_bytes = h.storage == H3D_STORE_SKELETON
                           ? h.lu_off_total * (int64_t)sizeof(double) + h.sum_rank * (int64_t)sizeof(int)
                           : (h.u_elems + h.v_elems + h.sym_elems) * (int64_t)h.elem();
    st->near_interactions = h.near_interactions;
    st->device_bytes = (int64_t)h.mem.total();
    st->build_ms = h.build_ms;
    // vertex blocks: count on demand
    std::vector<unsigned char> cls((size_t)h.nblk);
    if (h.nblk > 0 && cudaMemcpy(cls.data(), h.blk_cls, (size_t)h.nblk, cudaMemcpyDeviceToHost) != cudaSuccess)
        return H3D_ERR_CUDA;
    st->n_vertex_blocks = std::count(cls.begin(), cls.end(), (unsigned char)3);
    return H3D_OK;
}

h3d_status h3d_export_tree(h3d_handle hh, int64_t *perm, uint64_t *keys, int *nbox, uint64_t *box_key,
                           int64_t *box_start, int64_t *box_end) {
    if (!hh || !perm || !keys || !nbox || !box_key || !box_start || !box_end) return H3D_ERR_ARG;
    const Handle &h = *hh->p;
    if (!h.ok) return H3D_ERR_STATE;
    return guard([&] {
        const size_t n = (size_t)h.N, nb = (size_t)h.n_boxes;
        std::vector<int> p(n), bs(nb), be(nb);
        H3D_CUDA(cudaMemcpy(p.data(), h.perm, n * sizeof(int), cudaMemcpyDeviceToHost));
        H3D_CUDA(cudaMemcpy(keys, h.keys, n * sizeof(uint64_t), cudaMemcpyDeviceToHost));
        H3D_CUDA(cudaMemcpy(box_key, h.box_key, nb * sizeof(uint64_t), cudaMemcpyDeviceToHost));
        H3D_CUDA(cudaMemcpy(bs.data(), h.box_start, nb * sizeof(int), cudaMemcpyDeviceToHost));
        H3D_CUDA(cudaMemcpy(be.data(), h.box_end, nb * sizeof(int), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) perm[i] = p[i];
        for (size_t i = 0; i < nb; ++i) { box_start[i] = bs[i]; box_end[i] = be[i]; }
        for (int l = 0; l <= h.L; ++l) nbox[l] = h.nbox[l];
    });
}

h3d_status h3d_export_lists(h3d_handle hh, int *blk_level, int *blk_tgt, int *blk_src, int *blk_cls, int *near_tgt,
                            int *near_src, int *near_cls) {
    if (!hh) return H3D_ERR_ARG;
    const Handle &h = *hh->p;
    if (!h.ok) return H3D_ERR_STATE;
    if (h.nblk > 0 && (!blk_level || !blk_tgt || !blk_src || !blk_cls)) return H3D_ERR_ARG;
    if (!near_tgt || !near_src || !near_cls) return H3D_ERR_ARG;
    return guard([&] {
        const size_t nb = (size_t)h.nblk, nn = (size_t)h.nnear;
        std::vector<unsigned char> lev(nb), cls(nb), ncl(nn);
        std::vector<int> nptr((size_t)h.nleaf + 1);
        if (nb > 0) {
            H3D_CUDA(cudaMemcpy(lev.data(), h.blk_lev, nb, cudaMemcpyDeviceToHost));
            H3D_CUDA(cudaMemcpy(cls.data(), h.blk_cls, nb, cudaMemcpyDeviceToHost));
            H3D_CUDA(cudaMemcpy(blk_tgt, h.blk_tgt, nb * sizeof(int), cudaMemcpyDeviceToHost));
            H3D_CUDA(cudaMemcpy(blk_src, h.blk_src, nb * sizeof(int), cudaMemcpyDeviceToHost));
        }
        for (size_t b = 0; b < nb; ++b) {
            blk_level[b] = lev[b];
            blk_cls[b] = cls[b];
            blk_tgt[b] -= (int)h.box_off[lev[b]];
            blk_src[b] -= (int)h.box_off[lev[b]];
        }
        H3D_CUDA(cudaMemcpy(nptr.data(), h.near_ptr, nptr.size() * sizeof(int), cudaMemcpyDeviceToHost));
        H3D_CUDA(cudaMemcpy(near_src, h.near_src, nn * sizeof(int), cudaMemcpyDeviceToHost));
        H3D_CUDA(cudaMemcpy(ncl.data(), h.near_cls, nn, cudaMemcpyDeviceToHost));
        for (int z = 0; z < h.nleaf; ++z)
            for (int p = nptr[z]; p < nptr[z + 1]; ++p) near_tgt[p] = z;
        for (size_t p = 0; p < nn; ++p) near_cls[p] = ncl[p];
    });
}

h3d_status h3d_export_pivots(h3d_handle hh, int *rank, int *sigma, int *tau) {
    if (!hh) return H3D_ERR_ARG;
    const Handle &h = *hh->p;
    if (!h.ok) return H3D_ERR_STATE;
    if ((h.nblk > 0 && !rank) || (h.sum_rank > 0 && (!sigma || !tau))) return H3D_ERR_ARG;
    return guard([&] {
        if (h.nblk > 0) H3D_CUDA(cudaMemcpy(rank, h.rank, (size_t)h.nblk * sizeof(int), cudaMemcpyDeviceToHost));
        if (h.sum_rank > 0) {
            H3D_CUDA(cudaMemcpy(sigma, h.sigma, (size_t)h.sum_rank * sizeof(int), cudaMemcpyDeviceToHost));
            H3D_CUDA(cudaMemcpy(tau, h.tau, (size_t)h.sum_rank * sizeof(int), cudaMemcpyDeviceToHost));
        }
    });
}

h3d_status h3d_import_pivots(h3d_handle hh, const int *rank, const int *sigma, const int *tau, void *stream) {
    if (!hh) return H3D_ERR_ARG;
    Handle &h = *hh->p;
    if (!h.ok) return H3D_ERR_STATE;
    if (h3d_status e = async_error(h)) return e;
    if (h.nblk > 0 && !rank) return H3D_ERR_ARG;
    int64_t total = 0;
    for (int64_t b = 0; b < h.nblk; ++b) {
        if (rank[b] < 0) return H3D_ERR_ARG;
        total += rank[b];
    }
    if (total > 0 && (!sigma || !tau)) return H3D_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    Handle *n = same_parameters(h);
    if (!n) return H3D_ERR_OOM;
    // the same points in the caller's order, from the handle's sorted copy: the
    // new build reproduces the tree and the lists bit for bit
    double *pts = nullptr;
    h3d_status st = guard([&] {
        H3D_CUDA(cudaStreamSynchronize(s));
        H3D_CUDA(cudaMalloc((void **)&pts, (size_t)h.N * 3 * sizeof(double)));
        h3d::unsorted_points(h, pts, s);
    });
    if (st == H3D_OK) {
        const h3d::FrozenPivots fp{rank, sigma, tau};
        st = build_into(*n, pts, s, &fp);
    }
    if (pts) cudaFree(pts);
    if (st != H3D_OK) {
        delete n;
        return st;
    }
    cudaDeviceSynchronize();   // nothing may still use the old handle's memory
    delete hh->p;
    hh->p = n;
    return H3D_OK;
}

h3d_status h3d_set_points(h3d_handle hh, const double *points, void *stream) {
    if (!hh || !points) return H3D_ERR_ARG;
    Handle &h = *hh->p;
    if (!h.ok) return H3D_ERR_STATE;
    if (h3d_status e = async_error(h)) return e;
    if (!is_device_ptr(points)) return H3D_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    const h3d_status st = guard([&] {
        h3d::Arena tmp;
        if (!h3d::update_points(h, points, s, tmp)) return;   // the same coordinates: nothing to re-form
        if (h.storage == H3D_STORE_SKELETON) h3d::refactor_skeleton(h, s);
        else h3d::reform_factors(h, s, tmp);
        H3D_CUDA(cudaStreamSynchronize(s));
    });
    if (st != H3D_OK && st != H3D_ERR_DOMAIN) h.ok = false;   // factors may be half re-formed
    return st;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of independent operators (many point clouds), one right-hand side
// each.  Two ways to run them:
//   persistent  one launch of the persistent multi-operator kernel
//               (h3d_batch.cu), in a CUDA graph with the reset of its queue;
//               available when every handle stores factors and all are FP32
//               (or all FP64);
//   graph       each handle's own kernels captured once into a CUDA graph
//               whose branches (one stream each) run the clouds side by side;
//               later calls with the same vectors replay it with one launch.
struct h3d_batch_s {
    h3d::BatchPlan *plan = nullptr;               // persistent form, if available
    bool persistent = false;
    int ctas_per_sm = 0;
    std::vector<h3d_handle> hs;
    std::vector<int64_t> cost;                    // per handle: factor entries + near interactions
    int branches = 0;                             // streams in the graph
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> st;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t exec = nullptr;
    int exec_branches = 0;
    std::vector<const void *> xs;
    std::vector<void *> ys;
    ~h3d_batch_s() {
        h3d::batch_plan_free(plan);
        if (exec) cudaGraphExecDestroy(exec);
        for (cudaEvent_t e : join) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        for (cudaStream_t s : st) cudaStreamDestroy(s);
        if (cap) cudaStreamDestroy(cap);
    }
};

namespace {

// longest job first onto the least loaded branch
std::vector<int> assign_branches(const std::vector<int64_t> &cost, int nb) {
    std::vector<int> order(cost.size()), owner(cost.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b] || (cost[a] == cost[b] && a < b); });
    std::vector<int64_t> load(nb, 0);
    for (int i : order) {
        const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        owner[i] = b;
        load[b] += cost[i];
    }
    return owner;
}

void batch_capture(h3d_batch_s &B, const void *const *x, void *const *y, int nb) {
    if (B.exec) {
        H3D_CUDA(cudaGraphExecDestroy(B.exec));
        B.exec = nullptr;
    }
    while ((int)B.st.size() < nb) {
        cudaStream_t s;
        cudaEvent_t e;
        H3D_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        H3D_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        B.st.push_back(s);
        B.join.push_back(e);
    }
    const std::vector<int> owner = assign_branches(B.cost, nb);
    cudaGraph_t g = nullptr;
    H3D_CUDA(cudaStreamBeginCapture(B.cap, cudaStreamCaptureModeThreadLocal));
    try {
        H3D_CUDA(cudaEventRecord(B.fork, B.cap));
        for (int b = 0; b < nb; ++b) H3D_CUDA(cudaStreamWaitEvent(B.st[b], B.fork, 0));
        for (size_t i = 0; i < B.hs.size(); ++i) h3d::run_matvec(*B.hs[i]->p, x[i], y[i], 1, false, B.st[owner[i]]);
        for (int b = 0; b < nb; ++b) {
            H3D_CUDA(cudaEventRecord(B.join[b], B.st[b]));
            H3D_CUDA(cudaStreamWaitEvent(B.cap, B.join[b], 0));
        }
    } catch (...) {
        cudaStreamEndCapture(B.cap, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    H3D_CUDA(cudaStreamEndCapture(B.cap, &g));
    const cudaError_t e = cudaGraphInstantiate(&B.exec, g, 0);
    cudaGraphDestroy(g);
    H3D_CUDA(e);
    B.exec_branches = nb;
    B.xs.assign(x, x + B.hs.size());
    B.ys.assign(y, y + B.hs.size());
}

h3d_status batch_check(h3d_batch B, const void *const *x, void *const *y) {
    if (!B || !x || !y) return H3D_ERR_ARG;
    for (size_t i = 0; i < B->hs.size(); ++i) {
        const Handle &h = *B->hs[i]->p;
        if (!h.ok) return H3D_ERR_STATE;
        if (h3d_status e = async_error(h)) return e;
        if (!x[i] || !y[i] || x[i] == y[i]) return H3D_ERR_ARG;
    }
    return H3D_OK;
}

bool same_vectors(const h3d_batch_s &B, const void *const *x, void *const *y) {
    for (size_t i = 0; i < B.hs.size(); ++i)
        if (B.xs[i] != x[i] || B.ys[i] != y[i]) return false;
    return true;
}

// (size, rank) bucket of a handle for the per-bucket item shapes of the tuner:
// N below 2^15, below 2^17, or larger; largest rank up to 96 or above
int tune_bucket(const Handle &h) {
    const int sc = h.N < (1 << 15) ? 0 : h.N < (1 << 17) ? 1 : 2;
    const int rc = h.max_rank <= 96 ? 0 : 1;
    return 3 * rc + sc;
}

// persistent form: leaves per near-field / leaf item
constexpr int kDefaultNearGroup = 4, kDefaultLeafGroup = 2;   // (a near item gives each of 4 warps a leaf)
constexpr int kDefaultLag = 0;                                 // phase-major queue

void batch_run(h3d_batch_s &B, const void *const *x, void *const *y, cudaStream_t s) {
    if (B.persistent) {
        h3d::batch_plan_run(*B.plan, x, y, B.ctas_per_sm, s);
        return;
    }
    if (!B.exec || B.exec_branches != B.branches || !same_vectors(B, x, y)) batch_capture(B, x, y, B.branches);
    H3D_CUDA(cudaGraphLaunch(B.exec, s));
}

// mean time of three runs after one warm-up (synchronises s)
float batch_time(h3d_batch_s &B, const void *const *x, void *const *y, cudaStream_t s, cudaEvent_t e0,
                 cudaEvent_t e1) {
    batch_run(B, x, y, s);
    H3D_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < 3; ++r) batch_run(B, x, y, s);
    H3D_CUDA(cudaEventRecord(e1, s));
    H3D_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    H3D_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return ms / 3.f;
}

}  // namespace

extern "C" {

h3d_status h3d_batch_create(const h3d_handle *handles, int count, h3d_batch *out) {
    if (!handles || count < 1 || !out) return H3D_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        if (!handles[i] || !handles[i]->p->ok) return H3D_ERR_ARG;
        for (int j = 0; j < i; ++j)   // a handle's scratch serves one product at a time
            if (handles[j] == handles[i]) return H3D_ERR_ARG;
    }
    h3d_batch_s *B = new (std::nothrow) h3d_batch_s;
    if (!B) return H3D_ERR_OOM;
    const h3d_status st = guard([&] {
        B->hs.assign(handles, handles + count);
        for (int i = 0; i < count; ++i) {   // work estimate: factor entries plus the near field
            const Handle &h = *handles[i]->p;
            B->cost.push_back(h.factor_entries + h.N * 32);
        }
        B->branches = std::min(count, 8);
        H3D_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
        H3D_CUDA(cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming));
        std::vector<Handle *> hv;
        for (int i = 0; i < count; ++i) hv.push_back(handles[i]->p);
        B->plan = h3d::batch_plan_create(hv, kDefaultNearGroup, kDefaultLeafGroup, kDefaultLag);
        if (B->plan) {
            B->persistent = true;
            B->ctas_per_sm = h3d::batch_plan_max_ctas_per_sm(*B->plan);
        }
    });
    if (st != H3D_OK) {
        delete B;
        return st;
    }
    *out = B;
    return H3D_OK;
}

h3d_status h3d_batch_matvec(h3d_batch B, const void *const *x, void *const *y, void *stream) {
    if (h3d_status e = batch_check(B, x, y)) return e;
    return guard([&] { batch_run(*B, x, y, as_stream(stream)); });
}

h3d_status h3d_batch_tune(h3d_batch B, const void *const *x, void *const *y, void *stream, int *branches_out) {
    if (h3d_status e = batch_check(B, x, y)) return e;
    return guard([&] {
        cudaStream_t s = as_stream(stream);
        cudaEvent_t e0, e1;
        H3D_CUDA(cudaEventCreate(&e0));
        H3D_CUDA(cudaEventCreate(&e1));
        // graph form: 1, 2, 4, ... branches
        float best_graph = -1.f;
        int best_nb = 1;
        const int n = (int)B->hs.size();
        B->persistent = false;
        for (int nb = 1; nb <= std::min(n, 32); nb *= 2) {
            B->branches = nb;
            const float ms = batch_time(*B, x, y, s, e0, e1);
            if (best_graph < 0.f || ms < best_graph) {
                best_graph = ms;
                best_nb = nb;
            }
        }
        B->branches = best_nb;
        bool use_persistent = false;
        if (B->plan) {
            // persistent form, one item shape for every operator: leaves per item
            // x queue order x CTAs per SM
            const int cmax = h3d::batch_plan_max_ctas_per_sm(*B->plan);
            static const int groups[][2] = {{4, 1}, {4, 2}, {8, 4}};
            float best = -1.f;
            int best_cps = cmax, best_ng = kDefaultNearGroup, best_lg = kDefaultLeafGroup, best_lag = kDefaultLag;
            B->persistent = true;
            for (int lag : {0, 2, 8})
                for (const auto &g : groups) {
                    h3d::batch_plan_regroup(*B->plan, g[0], g[1], lag);
                    for (int cps : {cmax - 1, cmax}) {
                        if (cps < 1) continue;
                        B->ctas_per_sm = cps;
                        const float ms = batch_time(*B, x, y, s, e0, e1);
                        if (best < 0.f || ms < best) {
                            best = ms;
                            best_cps = cps;
                            best_ng = g[0];
                            best_lg = g[1];
                            best_lag = lag;
                        }
                    }
                }
            // then the item shape per (size, rank) bucket of operators, one
            // bucket at a time (coordinate descent from the common best)
            B->ctas_per_sm = best_cps;
            std::vector<int> ngv(n, best_ng), lgv(n, best_lg), bucket(n);
            for (int i = 0; i < n; ++i) bucket[i] = tune_bucket(*B->hs[i]->p);
            static const int cand[][2] = {{2, 1}, {4, 1}, {4, 2}, {8, 2}, {8, 4}, {16, 4}};
            for (int k = 0; k < 6; ++k) {
                if (std::find(bucket.begin(), bucket.end(), k) == bucket.end()) continue;
                int bng = best_ng, blg = best_lg;
                for (int i = 0; i < n; ++i)
                    if (bucket[i] == k) { bng = ngv[i]; blg = lgv[i]; break; }
                for (const auto &c : cand) {
                    if (c[0] == bng && c[1] == blg) continue;
                    for (int i = 0; i < n; ++i)
                        if (bucket[i] == k) { ngv[i] = c[0]; lgv[i] = c[1]; }
                    h3d::batch_plan_set_groups(*B->plan, ngv.data(), lgv.data(), best_lag);
                    const float ms = batch_time(*B, x, y, s, e0, e1);
                    if (ms < best) {
                        best = ms;
                        bng = c[0];
                        blg = c[1];
                    }
                }
                for (int i = 0; i < n; ++i)
                    if (bucket[i] == k) { ngv[i] = bng; lgv[i] = blg; }
            }
            h3d::batch_plan_set_groups(*B->plan, ngv.data(), lgv.data(), best_lag);
            use_persistent = best < best_graph;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        B->persistent = use_persistent;
        if (!use_persistent) batch_capture(*B, x, y, best_nb);
        if (branches_out) *branches_out = use_persistent ? 0 : best_nb;
    });
}

h3d_status h3d_batch_groups(h3d_batch B, int *near_groups, int *leaf_groups) {
    if (!B || !B->plan) return H3D_ERR_ARG;
    h3d::batch_plan_op_groups(*B->plan, near_groups, leaf_groups);
    return H3D_OK;
}

h3d_status h3d_batch_configure(h3d_batch B, int persistent, int ctas_per_sm, int near_group, int leaf_group, int lag) {
    if (!B || (persistent && !B->plan) || ctas_per_sm < 0 || near_group < 0 || leaf_group < 0 || lag < -1)
        return H3D_ERR_ARG;
    B->persistent = persistent != 0;
    if (!B->plan) return H3D_OK;
    return guard([&] {
        if (ctas_per_sm > 0) B->ctas_per_sm = std::min(ctas_per_sm, h3d::batch_plan_max_ctas_per_sm(*B->plan));
        int ng = 0, lg = 0, lo = 0;
        h3d::batch_plan_groups(*B->plan, &ng, &lg, &lo);
        const int ng2 = near_group > 0 ? near_group : ng, lg2 = leaf_group > 0 ? leaf_group : lg,
                  lo2 = lag >= 0 ? lag : lo;
        if (ng2 != ng || lg2 != lg || lo2 != lo) h3d::batch_plan_regroup(*B->plan, ng2, lg2, lo2);
    });
}

h3d_status h3d_batch_set_wait_limit(h3d_batch B, int64_t ns) {
    if (!B || ns < 1000 || ns > (int64_t)60 * 1000000000LL) return H3D_ERR_ARG;
    if (!B->plan) return H3D_OK;
    return guard([&] { h3d::batch_plan_set_wait(*B->plan, (long long)ns); });
}

h3d_status h3d_batch_set_queue(h3d_batch B, const int *items, int64_t count) {
    if (!B || !B->plan || (items && count < 1) || count < 0) return H3D_ERR_ARG;
    h3d_status st = H3D_OK;
    const h3d_status g = guard([&] {
        if (!h3d::batch_plan_set_queue(*B->plan, items, count)) st = H3D_ERR_ARG;
    });
    return g != H3D_OK ? g : st;
}

h3d_status h3d_batch_get_queue(h3d_batch B, int *items, int64_t cap, int64_t *count) {
    if (!B || !B->plan || !count || cap < 0) return H3D_ERR_ARG;
    h3d::batch_plan_get_queue(*B->plan, nullptr, 0, count);
    if (items && cap < *count) return H3D_ERR_ARG;
    if (items) h3d::batch_plan_get_queue(*B->plan, items, cap, count);
    return H3D_OK;
}

h3d_status h3d_batch_info(h3d_batch B, int *persistent, int *ctas_per_sm, int *branches) {
    if (!B) return H3D_ERR_ARG;
    if (persistent) *persistent = B->persistent ? 1 : B->plan ? 0 : -1;
    if (ctas_per_sm) *ctas_per_sm = B->ctas_per_sm;
    if (branches) *branches = B->branches;
    return H3D_OK;
}

h3d_status h3d_batch_free(h3d_batch B) {
    if (!B) return H3D_OK;
    cudaDeviceSynchronize();
    delete B;
    return H3D_OK;
}

}  // extern "C"
