// h3d_stream.cuh -- device building blocks of the single-column HODLR3D
// product (Alg. 2), shared by the per-operator kernels (h3d_matvec.cu) and the
// persistent multi-operator kernel (h3d_batch.cu):
//   gather_task   A7: t_b = V_b^T xs(Y_b) over one row range of a source box
//   reduce_split  A7: sum of the row-range partials of a split source box
//   near_field    A6: the dense self / face / edge sum of one leaf
//   leaf_task     A8 + A9 (+ the leaf's near-field sum): y(Z) for one leaf Z
// Each function works on one work item with the whole CTA.  The CG template
// flag marks inputs that may have been written earlier in the same launch (t,
// partials, near sums): they are then never read through the read-only path
// (see ldx / ldr).
#pragma once

#include "h3d_async.cuh"
#include "h3d_internal.cuh"

namespace h3d {

namespace {
constexpr int kGatherThreads = 256;
constexpr int kLeafThreads = 128;
constexpr int kTaskMaxRows = 2048;   // rows of one gather task, at most

struct __align__(16) Pt4d {
    double x, y, z, w;
};
__device__ __forceinline__ Pt4d make_pt4d(double x, double y, double z, double w) { return Pt4d{x, y, z, w}; }

// Sum accumulator.  FP32 sums of hundreds of random-sign products lose about
// u*sqrt(n/2) relative accuracy when added in sequence, so FP32 uses a
// compensated (Kahan) sum; FP64 adds plainly.
template <class T> struct Acc;
template <> struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ float get() const { return s - c; }
};
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double get() const { return s; }
};

template <class T> struct Vec;
template <> struct Vec<float> {
    using type = float4;
    static constexpr int W = 4;
    __device__ static __forceinline__ void get(const float4 &v, float (&o)[4]) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
};
template <> struct Vec<double> {
    using type = double2;
    static constexpr int W = 2;
    __device__ static __forceinline__ void get(const double2 &v, double (&o)[2]) { o[0] = v.x; o[1] = v.y; }
};

template <class T>
__device__ __forceinline__ typename Vec<T>::type ld_stream(const T *p) {
    return __ldcs(reinterpret_cast<const typename Vec<T>::type *>(p));
}

// Loads of values that a kernel reads but does not write.  CG: another CTA may
// have written them earlier in the same launch, so never the read-only path;
// ldx then reads through L2 only (values read once), ldr through L1
// (ld.global.ca: values that neighbouring leaves read again).  A CG read comes
// after this CTA's acquire of the writer's completion counter.  Without CG,
// ldx is a plain load and ldr takes the read-only path.
template <bool CG, class T>
__device__ __forceinline__ T ldx(const T *p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}
template <bool CG, class T>
__device__ __forceinline__ T ldr(const T *p) {
    if constexpr (CG) return __ldca(p);
    else return __ldg(p);
}

// ---------------------------------------------------------------------------
// A7: T_Y = V_Y^T xs(Y) over rows [r0, r1) of Y
struct GatherArgs {
    const int4 *task;            // (box, row0, row1, direct?1:0)
    const int64_t *pbase;        // partial base per task
    const int *box_start, *Rv, *ldv;
    const int64_t *vbase, *vcol0, *map_v;
};

// One gather task (box Y, rows [r0, r1)) with NT threads, RU rows (a multiple
// of 4) loaded per thread before they are used.  xsm holds kTaskMaxRows
// values, red NT * Vec<T>::W values (shared memory).  xs: the sources in
// Morton order (CG: written earlier in the same launch).
template <class T, int NT, int RU, bool CG>
__device__ __forceinline__ void gather_task(const GatherArgs &G, int task_id, const T *__restrict__ V,
                                            const T *__restrict__ xs, T *__restrict__ t, T *__restrict__ partial,
                                            T *xsm, T *red) {
    constexpr int W = Vec<T>::W;
    const int4 task = G.task[task_id];
    const int Y = task.x, r0 = task.y, r1 = task.z;
    const int nrows = r1 - r0;
    const int ld = G.ldv[Y], RvY = G.Rv[Y];
    const int ncv = ld / W;
    const T *Vb = V + G.vbase[Y] + (int64_t)r0 * ld;
    const int ys = G.box_start[Y] + r0;
    for (int r = threadIdx.x; r < nrows; r += NT) xsm[r] = CG ? __ldcg(xs + ys + r) : xs[ys + r];
    __syncthreads();
    const bool direct = task.w != 0;
    const int64_t pb = G.pbase[task_id];
    const int64_t vc0 = G.vcol0[Y];
    if (ncv >= NT) {
        for (int cv = threadIdx.x; cv < ncv; cv += NT) {
            Acc<T> acc[W];
            const T *p = Vb + cv * W;
            int r = 0;
            for (; r + RU <= nrows; r += RU) {
                typename Vec<T>::type v[RU];
#pragma unroll
                for (int u = 0; u < RU; ++u) v[u] = ld_stream(p + (int64_t)(r + u) * ld);
#pragma unroll
                for (int u = 0; u < RU; u += 4) {
                    T a0[W], a1[W], a2[W], a3[W];
                    Vec<T>::get(v[u], a0); Vec<T>::get(v[u + 1], a1); Vec<T>::get(v[u + 2], a2); Vec<T>::get(v[u + 3], a3);
                    const T *xr = xsm + r + u;
#pragma unroll
                    for (int e = 0; e < W; ++e) acc[e].add(a0[e] * xr[0] + a1[e] * xr[1] + a2[e] * xr[2] + a3[e] * xr[3]);
                }
            }
            for (; r < nrows; ++r) {
                T a[W];
                Vec<T>::get(ld_stream(p + (int64_t)r * ld), a);
#pragma unroll
                for (int e = 0; e < W; ++e) acc[e].add(a[e] * xsm[r]);
            }
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const int c = cv * W + e;
                if (c < RvY) {
                    if (direct) t[G.map_v[vc0 + c]] = acc[e].get();
                    else partial[pb + c] = acc[e].get();
                }
            }
        }
        return;
    }
    // few columns: split the rows over G groups, reduce in shared memory
    const int Gn = NT / ncv;
    const int g = threadIdx.x / ncv, cv = threadIdx.x - g * ncv;
    Acc<T> acc[W];
    if (g < Gn) {
        const T *p = Vb + cv * W;
        int r = g;
        for (; r + (RU - 1) * Gn < nrows; r += RU * Gn) {
            typename Vec<T>::type v[RU];
#pragma unroll
            for (int u = 0; u < RU; ++u) v[u] = ld_stream(p + (int64_t)(r + u * Gn) * ld);
#pragma unroll
            for (int u = 0; u < RU; u += 4) {
                T a0[W], a1[W], a2[W], a3[W];
                Vec<T>::get(v[u], a0); Vec<T>::get(v[u + 1], a1); Vec<T>::get(v[u + 2], a2); Vec<T>::get(v[u + 3], a3);
                const T *xr = xsm + r + u * Gn;
#pragma unroll
                for (int e = 0; e < W; ++e)
                    acc[e].add(a0[e] * xr[0] + a1[e] * xr[Gn] + a2[e] * xr[2 * Gn] + a3[e] * xr[3 * Gn]);
            }
        }
        for (; r < nrows; r += Gn) {
            T a[W];
            Vec<T>::get(ld_stream(p + (int64_t)r * ld), a);
#pragma unroll
            for (int e = 0; e < W; ++e) acc[e].add(a[e] * xsm[r]);
        }
#pragma unroll
        for (int e = 0; e < W; ++e) red[g * ld + cv * W + e] = acc[e].get();
    }
    __syncthreads();
    for (int c = threadIdx.x; c < RvY; c += NT) {
        T s = 0;
        for (int q = 0; q < Gn; ++q) s += red[q * ld + c];
        if (direct) t[G.map_v[vc0 + c]] = s;
        else partial[pb + c] = s;
    }
}

struct SplitArgs {
    const int *box, *ntask;
    const int64_t *pbase;
    const int *Rv, *ldv;
    const int64_t *vcol0, *map_v;
};

// Sum of the partials of split source box number q (nthreads threads).
template <class T, bool CG>
__device__ __forceinline__ void reduce_split(const SplitArgs &S, int q, int nthreads, const T *__restrict__ partial,
                                             T *__restrict__ t) {
    const int Y = S.box[q], nt = S.ntask[q], ld = S.ldv[Y], R = S.Rv[Y];
    const int64_t pb = S.pbase[q], vc0 = S.vcol0[Y];
    for (int c = threadIdx.x; c < R; c += nthreads) {
        T s = 0;
        for (int k = 0; k < nt; ++k) s += ldx<CG>(partial + pb + (int64_t)k * ld + c);
        t[S.map_v[vc0 + c]] = s;
    }
}

// ---------------------------------------------------------------------------
// near field helpers: stage one source leaf, accumulate over it.
struct LeafArgs {
    int L, nleaf, kind;
    double kappa, hL;
    int64_t offL;
    const int *box_start, *box_end, *perm, *leaf_ld, *leaf_anc, *R, *leaf_lo;
    const int64_t *leaf_lp, *ubase, *tbase;
    const int *near_ptr, *near_src;
    const unsigned char *near_dir;
    const float4 *ploc, *ploc_lo;
    const double *px, *py, *pz;
    // transpose
    const int *Rv, *ldv;
    const int64_t *vbase, *vcol0, *map_v, *tp_base;
    int *err;                         // device-visible error word (bounded waits that gave up)
};

// The near-field and leaf arguments of a built handle.
inline LeafArgs leaf_args(const Handle &h) {
    LeafArgs A{};
    A.L = h.L; A.nleaf = h.nleaf; A.kind = h.kernel; A.kappa = h.kappa;
    A.hL = h.side / (double)(1 << h.L);
    A.offL = h.box_off[h.L];
    A.box_start = h.box_start; A.box_end = h.box_end; A.perm = h.perm; A.leaf_ld = h.leaf_ld;
    A.leaf_anc = h.leaf_anc; A.R = h.R; A.leaf_lo = h.box_leaf_lo;
    A.leaf_lp = h.leaf_lp; A.ubase = h.ubase; A.tbase = h.tbase;
    A.near_ptr = h.near_ptr; A.near_src = h.near_src; A.near_dir = h.near_dir;
    A.ploc = h.ploc; A.ploc_lo = h.ploc_lo; A.px = h.px; A.py = h.py; A.pz = h.pz;
    A.Rv = h.Rv; A.ldv = h.ldv; A.vbase = h.vbase; A.vcol0 = h.vcol0; A.map_v = h.map_v; A.tp_base = h.tp_base;
    A.err = h.d_async_err;
    return A;
}

// Near-field sum for targets of leaf z: out[i] = sum over near leaves of
// K(i,j) xs_j (i in [0, m)).  Thread layout: S source groups x m targets.

// Source points of consecutive near leaves are staged together until the
// staging buffer (kMaxLeaf points) is full, so a CTA synchronises about
// (sum of near-leaf sizes) / kMaxLeaf times instead of once per near leaf.
__device__ void near_field(const LeafArgs &A, int z, int zs, int m, const float *__restrict__ xs, float *outsm,
                           float4 *srcf, Pt4d *, float *partsm) {
    // Coordinates are offsets from the leaf centre split into hi + lo floats.
    // A source point is moved into the target leaf's frame by the exact box
    // offset shift = (c_Y - c_Z); Fast2Sum keeps the rounding error of hi +
    // shift (|shift| >= |hi|), so differences keep full FP32 relative accuracy
    // even for very close pairs.
    const int T_ = kLeafThreads;
    const int S = m <= T_ ? max(1, T_ / m) : 1;
    const int ntg = m <= T_ ? 1 : (m + T_ - 1) / T_;   // targets per thread when m > T
    const int s = m <= T_ ? threadIdx.x / m : 0;
    const int i0 = m <= T_ ? threadIdx.x - s * m : threadIdx.x;
    const bool active = m <= T_ ? (s < S) : true;
    Acc<float> acc[4];
    float4 th[4], tl[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + q * T_;
        const bool ok = active && q < ntg && i < m;
        th[q] = ok ? A.ploc[zs + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        tl[q] = ok ? A.ploc_lo[zs + i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float kap = (float)A.kappa;
    const int p1 = A.near_ptr[z + 1];
    int p = A.near_ptr[z];
    while (p < p1) {
        // stage near leaves [p, pe) together
        int pe = p, cnt = 0;
        while (pe < p1) {
            const int y = A.near_src[pe];
            const int n = A.box_end[A.offL + y] - A.box_start[A.offL + y];
            if (cnt + n > kMaxLeaf && cnt > 0) break;
            cnt += n;
            ++pe;
        }
        __syncthreads();
        int base = 0;
        for (int q = p; q < pe; ++q) {
            const int y = A.near_src[q];
            const int ys = A.box_start[A.offL + y], n = A.box_end[A.offL + y] - ys;
            const int d = A.near_dir[q];
            const float sx = (float)((d / 9 - 1) * A.hL), sy = (float)(((d / 3) % 3 - 1) * A.hL),
                        sz = (float)((d % 3 - 1) * A.hL);
            for (int j = threadIdx.x; j < n; j += T_) {
                const float4 h = A.ploc[ys + j], l = A.ploc_lo[ys + j];
                const float hx = h.x + sx, hy = h.y + sy, hz = h.z + sz;
                const float ex = h.x - (hx - sx), ey = h.y - (hy - sy), ez = h.z - (hz - sz);
                srcf[2 * (base + j)] = make_float4(hx, hy, hz, xs[ys + j]);
                srcf[2 * (base + j) + 1] = make_float4(ex + l.x, ey + l.y, ez + l.z, 0.f);
            }
            base += n;
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + q * T_;
                if (q >= ntg || i >= m) break;
                auto term = [&](int j) {
                    const float4 sh = srcf[2 * j], sl = srcf[2 * j + 1];
                    const float dx = (th[q].x - sh.x) + (tl[q].x - sl.x);
                    const float dy = (th[q].y - sh.y) + (tl[q].y - sl.y);
                    const float dz = (th[q].z - sh.z) + (tl[q].z - sl.z);
                    const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    return kernel_fast(A.kind, kap, d2) * sh.w;
                };
                int j = s;
                // four independent interactions per compensated add (ILP)
                for (; j + 3 * S < cnt; j += 4 * S) {
                    const float a0 = term(j), a1 = term(j + S), a2 = term(j + 2 * S), a3 = term(j + 3 * S);
                    acc[q].add((a0 + a1) + (a2 + a3));
                }
                for (; j < cnt; j += S) acc[q].add(term(j));
            }
        }
        p = pe;
    }
    // reduce over source groups
    __syncthreads();
    if (m <= T_) {
        if (active) partsm[threadIdx.x] = acc[0].get();
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += T_) {
            float v = 0.f;
            for (int g = 0; g < S; ++g) v += partsm[g * m + i];
            outsm[i] = v;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + q * T_;
            if (q < ntg && i < m) outsm[i] = acc[q].get();
        }
    }
    __syncthreads();
}

__device__ void near_field(const LeafArgs &A, int z, int zs, int m, const double *__restrict__ xs, double *outsm,
                           float4 *, Pt4d *srcd, double *partsm) {
    const int T_ = kLeafThreads;
    const int S = m <= T_ ? max(1, T_ / m) : 1;
    const int ntg = m <= T_ ? 1 : (m + T_ - 1) / T_;
    const int s = m <= T_ ? threadIdx.x / m : 0;
    const int i0 = m <= T_ ? threadIdx.x - s * m : threadIdx.x;
    const bool active = m <= T_ ? (s < S) : true;
    double acc[4] = {0, 0, 0, 0};
    double tx[4], ty[4], tz[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + q * T_;
        const bool ok = active && q < ntg && i < m;
        tx[q] = ok ? A.px[zs + i] : 0.0;
        ty[q] = ok ? A.py[zs + i] : 0.0;
        tz[q] = ok ? A.pz[zs + i] : 0.0;
    }
    const int p1 = A.near_ptr[z + 1];
    int p = A.near_ptr[z];
    while (p < p1) {
        int pe = p, cnt = 0;
        while (pe < p1) {
            const int y = A.near_src[pe];
            const int n = A.box_end[A.offL + y] - A.box_start[A.offL + y];
            if (cnt + n > kMaxLeaf && cnt > 0) break;
            cnt += n;
            ++pe;
        }
        __syncthreads();
        int base = 0;
        for (int q = p; q < pe; ++q) {
            const int y = A.near_src[q];
            const int ys = A.box_start[A.offL + y], n = A.box_end[A.offL + y] - ys;
            for (int j = threadIdx.x; j < n; j += T_)
                srcd[base + j] = make_pt4d(A.px[ys + j], A.py[ys + j], A.pz[ys + j], xs[ys + j]);
            base += n;
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + q * T_;
                if (q >= ntg || i >= m) break;
                double a = 0.0;
                for (int j = s; j < cnt; j += S) {
                    const Pt4d sp = srcd[j];
                    const double dx = tx[q] - sp.x, dy = ty[q] - sp.y, dz = tz[q] - sp.z;
                    const double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
                    a = fma(kernel_fast(A.kind, A.kappa, d2), sp.w, a);
                }
                acc[q] += a;
            }
        }
        p = pe;
    }
    __syncthreads();
    if (m <= T_) {
        if (active) partsm[threadIdx.x] = acc[0];
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += T_) {
            double v = 0.0;
            for (int g = 0; g < S; ++g) v += partsm[g * m + i];
            outsm[i] = v;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + q * T_;
            if (q < ntg && i < m) outsm[i] = acc[q];
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// A6 + A8 + A9: one CTA per leaf.
//
// Far field: for every level the leaf reads one contiguous U panel (ld x R_A,
// column-major).  The panels of all levels are cut into chunks of whole
// columns (<= kChunkBytes) and streamed through a ring of kStages shared-memory
// buffers by bulk asynchronous copies (TMA) that complete on one mbarrier per
// buffer; one elected thread issues the copies kStages-1 chunks ahead.  Threads
// own W consecutive rows of a column group and accumulate U(rows, c) t_A(c)
// from shared memory.  Then the near field and y = far + near in caller order.
constexpr int kStages = 4;
constexpr int kChunkBytes = 8192;
constexpr size_t kLeafDynSmem = (size_t)kStages * kChunkBytes;

struct ChunkPlan {
    const void *panel[kMaxDepth + 1];
    const void *tA[kMaxDepth + 1];
    int R[kMaxDepth + 1];
    int first[kMaxDepth + 2];   // first chunk of level l (l = 1..L), first[L+1] = total
};

template <class T>
__device__ __forceinline__ void chunk_of(const ChunkPlan &P, int L, int k, int cpc, int &l, int &c0, int &nc) {
    while (l < L && k >= P.first[l + 1]) ++l;
    c0 = (k - P.first[l]) * cpc;
    nc = min(cpc, P.R[l] - c0);
}

// One leaf Z with kLeafThreads threads.  stage: NS * kChunkBytes bytes of
// shared memory (128-byte aligned); bars: NS mbarriers initialised with an
// arrival count of 1; ring: the number of chunks this CTA has already taken
// through the ring (the buffer and phase of every later chunk follow from it;
// advanced here).  nearbuf may be null (far field only).  Returns false, with the error word set, when a copy did not
// arrive in time; no copy is then left in flight.
template <class T, bool CG, int NS = kStages>
__device__ __forceinline__ bool leaf_task(const LeafArgs &A, int z, const T *__restrict__ U, const T *__restrict__ t,
                                          const T *__restrict__ nearbuf, T *__restrict__ y, unsigned char *stage,
                                          uint64_t *bars, ChunkPlan &P, T *red, uint32_t &ring) {
    constexpr int W = Vec<T>::W;
    const int Zg = (int)(A.offL + z);
    const int zs = A.box_start[Zg], m = A.box_end[Zg] - zs;
    const int ld = A.leaf_ld[z];
    const int nr = ld / W;
    const int cpc = kChunkBytes / (ld * (int)sizeof(T));   // columns per chunk (ld <= 512)
    const int L = A.L;

    // per-level panels, one thread per level, then the chunk prefix
    if (threadIdx.x >= 1 && threadIdx.x <= L) {
        const int l = threadIdx.x;
        const int Ag = A.leaf_anc[(int64_t)(l - 1) * A.nleaf + z];
        const int RA = A.R[Ag];
        P.panel[l] = U + A.ubase[Ag] + (A.leaf_lp[z] - A.leaf_lp[A.leaf_lo[Ag]]) * RA;
        P.tA[l] = t + A.tbase[Ag];
        P.R[l] = RA;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int l = 1; l <= L; ++l) {
            P.first[l] = acc;
            acc += (P.R[l] + cpc - 1) / cpc;
        }
        P.first[L + 1] = acc;
    }
    __syncthreads();
    const int nchunks = P.first[L + 1];
    const uint32_t r0 = ring;

    // one elected thread keeps the ring full
    int pl = 1;
    auto issue = [&](int k) {
        int c0, nc;
        chunk_of<T>(P, L, k, cpc, pl, c0, nc);
        const uint32_t bytes = (uint32_t)(nc * ld * (int)sizeof(T));
        const uint32_t slot = (r0 + (uint32_t)k) % NS;
        mbar_arrive_expect_tx(&bars[slot], bytes);
        bulk_copy_g2s(stage + (size_t)slot * kChunkBytes, static_cast<const T *>(P.panel[pl]) + (int64_t)c0 * ld,
                      bytes, &bars[slot]);
    };
    auto wait = [&](int k) {
        const uint32_t q = r0 + (uint32_t)k;
        return mbar_wait(&bars[q % NS], (q / NS) & 1u);
    };
    if (threadIdx.x == 0)
        for (int k = 0; k < min(NS - 1, nchunks); ++k) issue(k);

    const int Gc = nr <= kLeafThreads ? kLeafThreads / nr : 1;
    const int g = nr <= kLeafThreads ? threadIdx.x / nr : 0;
    const int rv0 = nr <= kLeafThreads ? threadIdx.x - g * nr : threadIdx.x;
    Acc<T> acc[2][W];
    int cl_level = 1;
    for (int k = 0; k < nchunks; ++k) {
        const bool ok = wait(k);
        // every thread has finished chunk k-1 here, so its buffer may be refilled
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                *A.err = H3D_ERR_TIMEOUT;
                for (int j = k; j < min(k + NS - 1, nchunks); ++j) wait(j);   // copies still in flight
            }
            return false;
        }
        if (threadIdx.x == 0 && k + NS - 1 < nchunks) issue(k + NS - 1);
        int c0, nc;
        chunk_of<T>(P, L, k, cpc, cl_level, c0, nc);
        const T *sm = reinterpret_cast<const T *>(stage + (size_t)((r0 + (uint32_t)k) % NS) * kChunkBytes);
        const T *tA = static_cast<const T *>(P.tA[cl_level]) + c0;
        if (g < Gc) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int rv = rv0 + h * kLeafThreads;
                if (rv >= nr) break;
                const T *p = sm + rv * W;
                int c = g;
                for (; c + 3 * Gc < nc; c += 4 * Gc) {
                    typename Vec<T>::type v0 = *reinterpret_cast<const typename Vec<T>::type *>(p + c * ld),
                                          v1 = *reinterpret_cast<const typename Vec<T>::type *>(p + (c + Gc) * ld),
                                          v2 = *reinterpret_cast<const typename Vec<T>::type *>(p + (c + 2 * Gc) * ld),
                                          v3 = *reinterpret_cast<const typename Vec<T>::type *>(p + (c + 3 * Gc) * ld);
                    const T t0 = ldr<CG>(tA + c), t1 = ldr<CG>(tA + c + Gc), t2 = ldr<CG>(tA + c + 2 * Gc),
                            t3 = ldr<CG>(tA + c + 3 * Gc);
                    T a0[W], a1[W], a2[W], a3[W];
                    Vec<T>::get(v0, a0); Vec<T>::get(v1, a1); Vec<T>::get(v2, a2); Vec<T>::get(v3, a3);
#pragma unroll
                    for (int e = 0; e < W; ++e) acc[h][e].add(a0[e] * t0 + a1[e] * t1 + a2[e] * t2 + a3[e] * t3);
                }
                for (; c < nc; c += Gc) {
                    T a[W];
                    Vec<T>::get(*reinterpret_cast<const typename Vec<T>::type *>(p + c * ld), a);
                    const T tc = ldr<CG>(tA + c);
#pragma unroll
                    for (int e = 0; e < W; ++e) acc[h][e].add(a[e] * tc);
                }
            }
        }
    }
    ring = r0 + (uint32_t)nchunks;
    // reduce over column groups, add the near field, write in the caller's order
    if (Gc > 1) {
        if (g < Gc)
#pragma unroll
            for (int e = 0; e < W; ++e) red[g * ld + rv0 * W + e] = acc[0][e].get();
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += kLeafThreads) {
            T v = 0;
            for (int q = 0; q < Gc; ++q) v += red[q * ld + i];
            y[A.perm[zs + i]] = v + (nearbuf ? ldx<CG>(nearbuf + zs + i) : T(0));
        }
    } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int rv = rv0 + h * kLeafThreads;
            if (rv < nr)
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    const int i = rv * W + e;
                    if (i < m) y[A.perm[zs + i]] = acc[h][e].get() + (nearbuf ? ldx<CG>(nearbuf + zs + i) : T(0));
                }
        }
    }
    return true;
}

// A6 for leaf z with ONE warp (the warps of a CTA work on different leaves,
// with no CTA-wide barrier between them).  Lane l holds the targets
// i0 + l + 32q (q < kNearWarpTq, as many as the leaf has; larger leaves take
// several passes).  The sources of all near
// leaves are taken as one sequence: wpre[k] (per-warp shared memory, room for
// kNearWarpLists + 1 ints) holds the position of near leaf k in it, and each
// round stages the next kNearWarpSrc positions in the warp's buffer wsrc, every
// lane loading four positions at once.  xs (Morton order) was written earlier
// in the same launch: read through L2.  FP32: offsets from the leaf centre as
// hi + lo floats moved into the target leaf's frame as in near_field;
// compensated sums, four sources per added term.  Writes nearbuf.
constexpr int kNearWarpSrc = 128;
constexpr int kNearWarpTq = 2;        // target slots per lane
constexpr int kNearWarpLists = 27;    // near leaves per leaf at most: the leaf and its 26 neighbours

// position s of the source sequence -> near-list entry (binary search in wpre)
__device__ __forceinline__ int near_entry(const int *wpre, int nl, int s) {
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (wpre[mid] <= s) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// prefix of the near-leaf sizes into wpre[0..nl]; returns the total
__device__ __forceinline__ int near_prefix(const LeafArgs &A, int p0, int nl, int *wpre) {
    const int lane = threadIdx.x & 31;
    int carry = 0;
    for (int k0 = 0; k0 < nl; k0 += 32) {
        const int k = k0 + lane;
        int n = 0;
        if (k < nl) {
            const int y = A.near_src[p0 + k];
            n = A.box_end[A.offL + y] - A.box_start[A.offL + y];
        }
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (k < nl) wpre[k] = carry + incl - n;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) wpre[nl] = carry;
    __syncwarp();
    return carry;
}

__device__ __forceinline__ void near_warp(const LeafArgs &A, int z, const float *__restrict__ xs,
                                          float *__restrict__ nearbuf, float4 *wsrc, int *wpre) {
    const int lane = threadIdx.x & 31;
    const int Zg = (int)(A.offL + z);
    const int zs = A.box_start[Zg], m = A.box_end[Zg] - zs;
    const float kap = (float)A.kappa;
    const int p0 = A.near_ptr[z], nl = A.near_ptr[z + 1] - p0;
    const int total = near_prefix(A, p0, nl, wpre);
    for (int i0 = 0; i0 < m; i0 += 32 * kNearWarpTq) {
        const int nq = min(kNearWarpTq, (m - i0 + 31) >> 5);   // target slots in use (warp-uniform)
        float4 th[kNearWarpTq], tl[kNearWarpTq];
        Acc<float> acc[kNearWarpTq];
#pragma unroll
        for (int q = 0; q < kNearWarpTq; ++q) {
            const int i = i0 + lane + 32 * q;
            const bool ok = i < m;
            th[q] = ok ? A.ploc[zs + i] : make_float4(0.f, 0.f, 0.f, 0.f);
            tl[q] = ok ? A.ploc_lo[zs + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int s0 = 0; s0 < total; s0 += kNearWarpSrc) {
            const int cnt = min(kNearWarpSrc, total - s0);
            __syncwarp();   // the previous round's sources are consumed
#pragma unroll
            for (int k0 = 0; k0 < 4; k0 += 2) {   // two positions per lane at a time: locate, load, store
                int g[2], d[2];
                float4 h[2], l[2];
                float v[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int s = s0 + lane + 32 * (k0 + k);
                    g[k] = -1;
                    d[k] = 13;
                    if (s < s0 + cnt) {
                        const int e = near_entry(wpre, nl, s);
                        g[k] = A.box_start[A.offL + A.near_src[p0 + e]] + (s - wpre[e]);
                        d[k] = A.near_dir[p0 + e];
                    }
                }
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    if (g[k] >= 0) {
                        h[k] = A.ploc[g[k]];
                        l[k] = A.ploc_lo[g[k]];
                        v[k] = __ldcg(xs + g[k]);
                    }
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    if (g[k] >= 0) {
                        const float sx = (float)((d[k] / 9 - 1) * A.hL), sy = (float)(((d[k] / 3) % 3 - 1) * A.hL),
                                    sz = (float)((d[k] % 3 - 1) * A.hL);
                        const float hx = h[k].x + sx, hy = h[k].y + sy, hz = h[k].z + sz;
                        const float ex = h[k].x - (hx - sx), ey = h[k].y - (hy - sy), ez = h[k].z - (hz - sz);
                        const int j = lane + 32 * (k0 + k);
                        wsrc[2 * j] = make_float4(hx, hy, hz, v[k]);
                        wsrc[2 * j + 1] = make_float4(ex + l[k].x, ey + l[k].y, ez + l[k].z, 0.f);
                    }
            }
            __syncwarp();
            auto term = [&](int q, int j) {
                const float4 sh = wsrc[2 * j], sl = wsrc[2 * j + 1];
                const float dx = (th[q].x - sh.x) + (tl[q].x - sl.x);
                const float dy = (th[q].y - sh.y) + (tl[q].y - sl.y);
                const float dz = (th[q].z - sh.z) + (tl[q].z - sl.z);
                const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                return kernel_fast(A.kind, kap, d2) * sh.w;
            };
            int j = 0;
            for (; j + 4 <= cnt; j += 4)
#pragma unroll
                for (int q = 0; q < kNearWarpTq; ++q)
                    if (q < nq) acc[q].add((term(q, j) + term(q, j + 1)) + (term(q, j + 2) + term(q, j + 3)));
            for (; j < cnt; ++j)
#pragma unroll
                for (int q = 0; q < kNearWarpTq; ++q)
                    if (q < nq) acc[q].add(term(q, j));
        }
#pragma unroll
        for (int q = 0; q < kNearWarpTq; ++q) {
            const int i = i0 + lane + 32 * q;
            if (i < m) nearbuf[zs + i] = acc[q].get();
        }
        __syncwarp();   // wsrc is refilled by the next target group
    }
}

// FP64: global coordinates, plain sums.  wsrc holds kNearWarpSrc Pt4d.
__device__ __forceinline__ void near_warp(const LeafArgs &A, int z, const double *__restrict__ xs,
                                          double *__restrict__ nearbuf, Pt4d *wsrc, int *wpre) {
    const int lane = threadIdx.x & 31;
    const int Zg = (int)(A.offL + z);
    const int zs = A.box_start[Zg], m = A.box_end[Zg] - zs;
    const int p0 = A.near_ptr[z], nl = A.near_ptr[z + 1] - p0;
    const int total = near_prefix(A, p0, nl, wpre);
    for (int i0 = 0; i0 < m; i0 += 32 * kNearWarpTq) {
        const int nq = min(kNearWarpTq, (m - i0 + 31) >> 5);
        double tx[kNearWarpTq], ty[kNearWarpTq], tz[kNearWarpTq], acc[kNearWarpTq];
#pragma unroll
        for (int q = 0; q < kNearWarpTq; ++q) {
            acc[q] = 0.0;
            const int i = i0 + lane + 32 * q;
            const bool ok = i < m;
            tx[q] = ok ? A.px[zs + i] : 0.0;
            ty[q] = ok ? A.py[zs + i] : 0.0;
            tz[q] = ok ? A.pz[zs + i] : 0.0;
        }
        for (int s0 = 0; s0 < total; s0 += kNearWarpSrc) {
            const int cnt = min(kNearWarpSrc, total - s0);
            int g[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int s = s0 + lane + 32 * k;
                g[k] = -1;
                if (s < s0 + cnt) {
                    const int e = near_entry(wpre, nl, s);
                    g[k] = A.box_start[A.offL + A.near_src[p0 + e]] + (s - wpre[e]);
                }
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (g[k] >= 0) wsrc[lane + 32 * k] = make_pt4d(A.px[g[k]], A.py[g[k]], A.pz[g[k]], __ldcg(xs + g[k]));
            __syncwarp();
            for (int j = 0; j < cnt; ++j) {
                const Pt4d sp = wsrc[j];
#pragma unroll
                for (int q = 0; q < kNearWarpTq; ++q)
                    if (q < nq) {
                        const double dx = tx[q] - sp.x, dy = ty[q] - sp.y, dz = tz[q] - sp.z;
                        const double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
                        acc[q] = fma(kernel_fast(A.kind, A.kappa, d2), sp.w, acc[q]);
                    }
            }
        }
#pragma unroll
        for (int q = 0; q < kNearWarpTq; ++q) {
            const int i = i0 + lane + 32 * q;
            if (i < m) nearbuf[zs + i] = acc[q];
        }
        __syncwarp();
    }
}

// A6 for leaf z: the near-field sum into nearbuf (Morton order).  outsm holds
// kMaxLeaf values, partsm kLeafThreads, srcbuf kMaxLeaf * 32 bytes.
template <class T>
__device__ __forceinline__ void near_task(const LeafArgs &A, int z, const T *__restrict__ xs, T *__restrict__ nearbuf,
                                          T *outsm, T *partsm, unsigned char *srcbuf) {
    const int Zg = (int)(A.offL + z);
    const int zs = A.box_start[Zg], m = A.box_end[Zg] - zs;
    near_field(A, z, zs, m, xs, outsm, reinterpret_cast<float4 *>(srcbuf), reinterpret_cast<Pt4d *>(srcbuf),
                   partsm);
    for (int i = threadIdx.x; i < m; i += kLeafThreads) nearbuf[zs + i] = outsm[i];
}

}  // namespace

}  // namespace h3d
