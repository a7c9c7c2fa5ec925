// h3d_matvec.cu -- the HODLR3D matrix-vector product (Alg. 2) and its
// transpose on the GPU.
//
// Forward product y = A~ x, per right-hand side:
//   A5  xs = x[perm]                                  (k_permute_in)
//   A7  t_b = V_b^T xs(Y_b) for every block, grouped by source box Y: the
//       source box's V (n_Y x ldv_Y row-major) is streamed once with 128-bit
//       loads, threads over columns, rows split across tasks when Y is large
//       (partials reduced by k_reduce_partials)      (k_gather)
//   A6+A8+A9 one CTA per leaf Z: the dense self/face/edge near field with
//       kernel entries recomputed from staged source points, plus, for every
//       level, the panel of the ancestor's U restricted to Z's rows times the
//       ancestor's t; the sum is written straight to y in the caller's order
//                                                     (k_leaf)
// Transposed product y = A~^T x (the factor roles exchanged):
//   t'_b = U_b^T xs(X_b) per leaf panel, partials reduced per box
//                                                     (k_leafT_gather, k_reduceT)
//   per leaf: near field (K is symmetric, the near lists are symmetric) plus
//   V rows of every ancestor source box times t'       (k_leafT)
#include <algorithm>

#include "h3d_async.cuh"
#include "h3d_internal.cuh"

namespace h3d {

namespace {

constexpr int kGatherThreads = 256;
constexpr int kLeafThreads = 128;
constexpr int64_t kTaskElems = 1 << 18;   // factor entries streamed by one gather task
constexpr int kTaskMaxRows = 2048;

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

template <class T>
__global__ void k_permute_in(const T *__restrict__ x, const int *__restrict__ perm, int64_t n, T *__restrict__ xs) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) xs[i] = x[perm[i]];
}

// ---------------------------------------------------------------------------
// A7: T_Y = V_Y^T xs(Y) over rows [r0, r1) of Y
struct GatherArgs {
    const int4 *task;            // (box, row0, row1, direct?1:0)
    const int64_t *pbase;        // partial base per task
    const int *box_start, *Rv, *ldv;
    const int64_t *vbase, *vcol0, *map_v;
};

template <class T>
__global__ void __launch_bounds__(kGatherThreads) k_gather(GatherArgs G, const T *__restrict__ V,
                                                           const T *__restrict__ xs, T *__restrict__ t,
                                                           T *__restrict__ partial) {
    constexpr int W = Vec<T>::W;
    __shared__ T xsm[kTaskMaxRows];
    __shared__ T red[kGatherThreads * W];
    const int4 task = G.task[blockIdx.x];
    const int Y = task.x, r0 = task.y, r1 = task.z;
    const int nrows = r1 - r0;
    const int ld = G.ldv[Y], RvY = G.Rv[Y];
    const int ncv = ld / W;
    const T *Vb = V + G.vbase[Y] + (int64_t)r0 * ld;
    const int ys = G.box_start[Y] + r0;
    for (int r = threadIdx.x; r < nrows; r += kGatherThreads) xsm[r] = xs[ys + r];
    __syncthreads();
    const bool direct = task.w != 0;
    const int64_t pb = G.pbase[blockIdx.x];
    const int64_t vc0 = G.vcol0[Y];
    if (ncv >= kGatherThreads) {
        for (int cv = threadIdx.x; cv < ncv; cv += kGatherThreads) {
            Acc<T> acc[W];
            const T *p = Vb + cv * W;
            int r = 0;
            for (; r + 4 <= nrows; r += 4) {
                typename Vec<T>::type v0 = ld_stream(p + (int64_t)r * ld), v1 = ld_stream(p + (int64_t)(r + 1) * ld),
                                      v2 = ld_stream(p + (int64_t)(r + 2) * ld), v3 = ld_stream(p + (int64_t)(r + 3) * ld);
                T a0[W], a1[W], a2[W], a3[W];
                Vec<T>::get(v0, a0); Vec<T>::get(v1, a1); Vec<T>::get(v2, a2); Vec<T>::get(v3, a3);
#pragma unroll
                for (int e = 0; e < W; ++e)
                    acc[e].add(a0[e] * xsm[r] + a1[e] * xsm[r + 1] + a2[e] * xsm[r + 2] + a3[e] * xsm[r + 3]);
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
    const int Gn = kGatherThreads / ncv;
    const int g = threadIdx.x / ncv, cv = threadIdx.x - g * ncv;
    Acc<T> acc[W];
    if (g < Gn) {
        const T *p = Vb + cv * W;
        int r = g;
        for (; r + 3 * Gn < nrows; r += 4 * Gn) {
            typename Vec<T>::type v0 = ld_stream(p + (int64_t)r * ld), v1 = ld_stream(p + (int64_t)(r + Gn) * ld),
                                  v2 = ld_stream(p + (int64_t)(r + 2 * Gn) * ld),
                                  v3 = ld_stream(p + (int64_t)(r + 3 * Gn) * ld);
            T a0[W], a1[W], a2[W], a3[W];
            Vec<T>::get(v0, a0); Vec<T>::get(v1, a1); Vec<T>::get(v2, a2); Vec<T>::get(v3, a3);
#pragma unroll
            for (int e = 0; e < W; ++e)
                acc[e].add(a0[e] * xsm[r] + a1[e] * xsm[r + Gn] + a2[e] * xsm[r + 2 * Gn] + a3[e] * xsm[r + 3 * Gn]);
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
    for (int c = threadIdx.x; c < RvY; c += kGatherThreads) {
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

template <class T>
__global__ void k_reduce_partials(SplitArgs S, const T *__restrict__ partial, T *__restrict__ t) {
    const int q = blockIdx.x;
    const int Y = S.box[q], nt = S.ntask[q], ld = S.ldv[Y], R = S.Rv[Y];
    const int64_t pb = S.pbase[q], vc0 = S.vcol0[Y];
    for (int c = threadIdx.x; c < R; c += blockDim.x) {
        T s = 0;
        for (int k = 0; k < nt; ++k) s += partial[pb + (int64_t)k * ld + c];
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

// Near-field sum for targets of leaf z: out[i] = sum over near leaves of
// K(i,j) xs_j (i in [0, m)).  Thread layout: S source groups x m targets.
template <class T>
__device__ void near_field(const LeafArgs &A, int z, int zs, int m, const T *__restrict__ xs, T *outsm,
                           float4 *srcf, Pt4d *srcd, T *partsm);

// Source points of consecutive near leaves are staged together until the
// staging buffer (kMaxLeaf points) is full, so a CTA synchronises about
// (sum of near-leaf sizes) / kMaxLeaf times instead of once per near leaf.
template <>
__device__ void near_field<float>(const LeafArgs &A, int z, int zs, int m, const float *__restrict__ xs, float *outsm,
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

template <>
__device__ void near_field<double>(const LeafArgs &A, int z, int zs, int m, const double *__restrict__ xs,
                                   double *outsm, float4 *, Pt4d *srcd, double *partsm) {
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

template <class T>
__global__ void __launch_bounds__(kLeafThreads) k_leaf(LeafArgs A, const T *__restrict__ U, const T *__restrict__ t,
                                                       const T *__restrict__ nearbuf, T *__restrict__ y) {
    constexpr int W = Vec<T>::W;
    extern __shared__ __align__(128) unsigned char stage[];   // kStages * kChunkBytes
    __shared__ __align__(8) uint64_t bars[kStages];
    __shared__ ChunkPlan P;
    __shared__ T red[kLeafThreads * W];
    const int z = blockIdx.x;
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
    if (threadIdx.x == 0) {
        for (int q = 0; q < kStages; ++q) mbar_init(&bars[q], 1);
        mbar_fence_init();
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

    // one elected thread keeps the ring full
    int pl = 1;
    auto issue = [&](int k) {
        int c0, nc;
        chunk_of<T>(P, L, k, cpc, pl, c0, nc);
        const uint32_t bytes = (uint32_t)(nc * ld * (int)sizeof(T));
        uint64_t *bar = &bars[k % kStages];
        mbar_arrive_expect_tx(bar, bytes);
        bulk_copy_g2s(stage + (size_t)(k % kStages) * kChunkBytes,
                      static_cast<const T *>(P.panel[pl]) + (int64_t)c0 * ld, bytes, bar);
    };
    if (threadIdx.x == 0)
        for (int k = 0; k < min(kStages - 1, nchunks); ++k) issue(k);

    const int Gc = nr <= kLeafThreads ? kLeafThreads / nr : 1;
    const int g = nr <= kLeafThreads ? threadIdx.x / nr : 0;
    const int rv0 = nr <= kLeafThreads ? threadIdx.x - g * nr : threadIdx.x;
    Acc<T> acc[2][W];
    int cl_level = 1;
    for (int k = 0; k < nchunks; ++k) {
        const bool ok = mbar_wait(&bars[k % kStages], (uint32_t)((k / kStages) & 1));
        // every thread has finished chunk k-1 here, so its buffer may be refilled
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                *A.err = H3D_ERR_TIMEOUT;
                for (int j = k; j < min(k + kStages - 1, nchunks); ++j)   // copies still in flight
                    mbar_wait(&bars[j % kStages], (uint32_t)((j / kStages) & 1));
            }
            return;
        }
        if (threadIdx.x == 0 && k + kStages - 1 < nchunks) issue(k + kStages - 1);
        int c0, nc;
        chunk_of<T>(P, L, k, cpc, cl_level, c0, nc);
        const T *sm = reinterpret_cast<const T *>(stage + (size_t)(k % kStages) * kChunkBytes);
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
                    const T t0 = __ldg(tA + c), t1 = __ldg(tA + c + Gc), t2 = __ldg(tA + c + 2 * Gc),
                            t3 = __ldg(tA + c + 3 * Gc);
                    T a0[W], a1[W], a2[W], a3[W];
                    Vec<T>::get(v0, a0); Vec<T>::get(v1, a1); Vec<T>::get(v2, a2); Vec<T>::get(v3, a3);
#pragma unroll
                    for (int e = 0; e < W; ++e) acc[h][e].add(a0[e] * t0 + a1[e] * t1 + a2[e] * t2 + a3[e] * t3);
                }
                for (; c < nc; c += Gc) {
                    T a[W];
                    Vec<T>::get(*reinterpret_cast<const typename Vec<T>::type *>(p + c * ld), a);
                    const T tc = __ldg(tA + c);
#pragma unroll
                    for (int e = 0; e < W; ++e) acc[h][e].add(a[e] * tc);
                }
            }
        }
    }
    // reduce over column groups, add the near field, write in the caller's order
    if (Gc > 1) {
        if (g < Gc)
#pragma unroll
            for (int e = 0; e < W; ++e) red[g * ld + rv0 * W + e] = acc[0][e].get();
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += kLeafThreads) {
            T v = 0;
            for (int q = 0; q < Gc; ++q) v += red[q * ld + i];
            y[A.perm[zs + i]] = v + nearbuf[zs + i];
        }
    } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int rv = rv0 + h * kLeafThreads;
            if (rv < nr)
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    const int i = rv * W + e;
                    if (i < m) y[A.perm[zs + i]] = acc[h][e].get() + nearbuf[zs + i];
                }
        }
    }
}

// A6: dense self / face / edge near field into nearbuf (Morton order).  A
// persistent grid of kNearCtasPerSm CTAs per SM walks the leaves; it runs on a
// high-priority second stream next to the memory-bound source-side gather,
// taking only a few warp slots per SM so that both proceed together.
constexpr int kNearCtasPerSm = 2;

template <class T>
__global__ void __launch_bounds__(kLeafThreads) k_near(LeafArgs A, const T *__restrict__ xs, T *__restrict__ nearbuf) {
    __shared__ T outsm[kMaxLeaf];
    __shared__ T partsm[kLeafThreads];
    __shared__ __align__(16) unsigned char srcbuf[kMaxLeaf * 32];
    for (int z = blockIdx.x; z < A.nleaf; z += gridDim.x) {
        const int Zg = (int)(A.offL + z);
        const int zs = A.box_start[Zg], m = A.box_end[Zg] - zs;
        near_field<T>(A, z, zs, m, xs, outsm, reinterpret_cast<float4 *>(srcbuf), reinterpret_cast<Pt4d *>(srcbuf),
                      partsm);
        for (int i = threadIdx.x; i < m; i += kLeafThreads) nearbuf[zs + i] = outsm[i];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// transpose: t'_A = U_A^T xs(A), per leaf panel
template <class T>
__global__ void __launch_bounds__(kLeafThreads) k_leafT_gather(LeafArgs A, const T *__restrict__ U,
                                                               const T *__restrict__ xs, T *__restrict__ t,
                                                               T *__restrict__ tpart) {
    __shared__ T xsm[kMaxLeaf];
    const int z = blockIdx.x;
    const int Zg = (int)(A.offL + z);
    const int zs = A.box_start[Zg], m = A.box_end[Zg] - zs;
    const int ld = A.leaf_ld[z];
    for (int i = threadIdx.x; i < m; i += kLeafThreads) xsm[i] = xs[zs + i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kLeafThreads / 32;
    for (int l = 1; l <= A.L; ++l) {
        const int Ag = A.leaf_anc[(int64_t)(l - 1) * A.nleaf + z];
        const int RA = A.R[Ag];
        if (RA == 0) continue;
        const T *panel = U + A.ubase[Ag] + (A.leaf_lp[z] - A.leaf_lp[A.leaf_lo[Ag]]) * RA;
        T *out = (l == A.L) ? t + A.tbase[Ag] : tpart + A.tp_base[(int64_t)(l - 1) * A.nleaf + z];
        for (int c = warp; c < RA; c += nw) {
            const T *col = panel + (int64_t)c * ld;
            T s = 0;
            for (int i = lane; i < m; i += 32) s += __ldcs(col + i) * xsm[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) out[c] = s;
        }
    }
}

// sum the per-leaf partials of every box A above the leaf level
struct ReduceTArgs {
    const int *box;       // global box indices of levels 1..L-1 with R > 0
    const int *level;
    const int *R, *leaf_lo, *leaf_hi;
    const int64_t *tbase, *tp_base;
    int nleaf;
};

template <class T>
__global__ void k_reduceT(ReduceTArgs S, const T *__restrict__ tpart, T *__restrict__ t) {
    const int Ag = S.box[blockIdx.x];
    const int l = S.level[blockIdx.x];
    const int RA = S.R[Ag], z0 = S.leaf_lo[Ag], z1 = S.leaf_hi[Ag];
    const int64_t base = S.tp_base[(int64_t)(l - 1) * S.nleaf + z0];
    for (int c = threadIdx.x; c < RA; c += blockDim.x) {
        T s = 0;
        for (int z = z0; z < z1; ++z) s += tpart[base + (int64_t)(z - z0) * RA + c];
        t[S.tbase[Ag] + c] = s;
    }
}

// per leaf: rows of every ancestor source box's V times t', plus the near field
template <class T>
__global__ void __launch_bounds__(kLeafThreads) k_leafT(LeafArgs A, const T *__restrict__ V, const T *__restrict__ t,
                                                        const T *__restrict__ nearbuf, T *__restrict__ y) {
    __shared__ T outsm[kMaxLeaf];
    __shared__ T tsm[2048];
    const int z = blockIdx.x;
    const int Zg = (int)(A.offL + z);
    const int zs = A.box_start[Zg], m = A.box_end[Zg] - zs;
    for (int i = threadIdx.x; i < m; i += kLeafThreads) outsm[i] = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kLeafThreads / 32;
    for (int l = 1; l <= A.L; ++l) {
        const int Yg = A.leaf_anc[(int64_t)(l - 1) * A.nleaf + z];
        const int RvY = A.Rv[Yg];
        if (RvY == 0) continue;
        const int ld = A.ldv[Yg];
        const int64_t vc0 = A.vcol0[Yg];
        const T *rows = V + A.vbase[Yg] + (int64_t)(zs - A.box_start[Yg]) * ld;
        for (int c0 = 0; c0 < RvY; c0 += 2048) {
            const int nc = min(2048, RvY - c0);
            __syncthreads();
            for (int c = threadIdx.x; c < nc; c += kLeafThreads) tsm[c] = t[A.map_v[vc0 + c0 + c]];
            __syncthreads();
            for (int i = warp; i < m; i += nw) {
                const T *row = rows + (int64_t)i * ld + c0;
                T s = 0;
                for (int c = lane; c < nc; c += 32) s += __ldcs(row + c) * tsm[c];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) outsm[i] += s;
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += kLeafThreads) y[A.perm[zs + i]] = outsm[i] + nearbuf[zs + i];
}

// ===========================================================================
// Several right-hand sides: blocks of kNQ columns per pass over the factors.
// x, t, partials and the near field are point-major inside a block
// (value (i, q) at i * kNQ + q), so every factor element streamed from HBM
// feeds kNQ fused multiply-adds.  Leaves of up to kMaxLeafMR points.
constexpr int kNQ = 8;
constexpr int kMaxLeafMR = 256;
constexpr int kRowChunk = 256;

template <class T>
__global__ void k_permute_in_mr(const T *__restrict__ x, int64_t n, int q0, int nq, const int *__restrict__ perm,
                                T *__restrict__ xs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = perm[i];
#pragma unroll
    for (int q = 0; q < kNQ; ++q) xs[i * kNQ + q] = q < nq ? x[(int64_t)(q0 + q) * n + o] : T(0);
}

// T_Y(c, q) = sum_r V_Y(r, c) x(r, q) over the task's rows
template <class T>
__global__ void __launch_bounds__(kGatherThreads) k_gather_mr(GatherArgs G, const T *__restrict__ V,
                                                              const T *__restrict__ xs, T *__restrict__ t,
                                                              T *__restrict__ partial) {
    constexpr int W = Vec<T>::W;
    __shared__ T xsm[kRowChunk * kNQ];
    __shared__ T red[kGatherThreads * W];
    const int4 task = G.task[blockIdx.x];
    const int Y = task.x, r0 = task.y, r1 = task.z;
    const int nrows = r1 - r0;
    const int ld = G.ldv[Y], RvY = G.Rv[Y];
    const int ncv = ld / W;
    const T *Vb = V + G.vbase[Y] + (int64_t)r0 * ld;
    const int64_t ys = (int64_t)G.box_start[Y] + r0;
    const bool direct = task.w != 0;
    const int64_t pb = G.pbase[blockIdx.x];
    const int64_t vc0 = G.vcol0[Y];
    const bool wide = ncv >= kGatherThreads;
    const int Gn = wide ? 1 : kGatherThreads / ncv;
    const int g = wide ? 0 : threadIdx.x / ncv;
    for (int cvb = 0; cvb < (wide ? ncv : 1); cvb += kGatherThreads) {
        const int cv = wide ? cvb + threadIdx.x : threadIdx.x - g * ncv;
        const bool act = wide ? cv < ncv : g < Gn;
        Acc<T> acc[W][kNQ];
        for (int rc = 0; rc < nrows; rc += kRowChunk) {
            const int nr = min(kRowChunk, nrows - rc);
            __syncthreads();
            for (int e = threadIdx.x; e < nr * kNQ; e += kGatherThreads) xsm[e] = xs[(ys + rc) * kNQ + e];
            __syncthreads();
            if (act) {
                const T *p = Vb + (int64_t)rc * ld + cv * W;
                int r = g;
                // four rows per compensated add: 4 FMAs per (column, rhs), then one add
                for (; r + 3 * Gn < nr; r += 4 * Gn) {
                    T a0[W], a1[W], a2[W], a3[W];
                    Vec<T>::get(ld_stream(p + (int64_t)r * ld), a0);
                    Vec<T>::get(ld_stream(p + (int64_t)(r + Gn) * ld), a1);
                    Vec<T>::get(ld_stream(p + (int64_t)(r + 2 * Gn) * ld), a2);
                    Vec<T>::get(ld_stream(p + (int64_t)(r + 3 * Gn) * ld), a3);
                    const T *x0 = xsm + r * kNQ, *x1 = x0 + Gn * kNQ, *x2 = x1 + Gn * kNQ, *x3 = x2 + Gn * kNQ;
#pragma unroll
                    for (int q = 0; q < kNQ; ++q)
#pragma unroll
                        for (int e = 0; e < W; ++e)
                            acc[e][q].add(a0[e] * x0[q] + a1[e] * x1[q] + a2[e] * x2[q] + a3[e] * x3[q]);
                }
                for (; r < nr; r += Gn) {
                    T a[W];
                    Vec<T>::get(ld_stream(p + (int64_t)r * ld), a);
                    const T *xr = xsm + r * kNQ;
#pragma unroll
                    for (int q = 0; q < kNQ; ++q)
#pragma unroll
                        for (int e = 0; e < W; ++e) acc[e][q].add(a[e] * xr[q]);
                }
            }
        }
        if (wide) {
            if (act)
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    const int c = cv * W + e;
                    if (c < RvY) {
                        T *o = direct ? t + G.map_v[vc0 + c] * kNQ : partial + (pb + c) * kNQ;
#pragma unroll
                        for (int q = 0; q < kNQ; ++q) o[q] = acc[e][q].get();
                    }
                }
        } else {
            for (int q = 0; q < kNQ; ++q) {
                if (act)
#pragma unroll
                    for (int e = 0; e < W; ++e) red[g * ld + cv * W + e] = acc[e][q].get();
                __syncthreads();
                for (int c = threadIdx.x; c < RvY; c += kGatherThreads) {
                    T v = 0;
                    for (int u = 0; u < Gn; ++u) v += red[u * ld + c];
                    T *o = direct ? t + G.map_v[vc0 + c] * kNQ : partial + (pb + c) * kNQ;
                    o[q] = v;
                }
                __syncthreads();
            }
        }
    }
}

template <class T>
__global__ void k_reduce_partials_mr(SplitArgs S, const T *__restrict__ partial, T *__restrict__ t) {
    const int q = blockIdx.x;
    const int Y = S.box[q], nt = S.ntask[q], ld = S.ldv[Y], R = S.Rv[Y];
    const int64_t pb = S.pbase[q], vc0 = S.vcol0[Y];
    for (int e = threadIdx.x; e < R * kNQ; e += blockDim.x) {
        const int c = e / kNQ, j = e - c * kNQ;
        T v = 0;
        for (int k = 0; k < nt; ++k) v += partial[(pb + (int64_t)k * ld + c) * kNQ + j];
        t[S.map_v[vc0 + c] * kNQ + j] = v;
    }
}

// near field of one leaf for kNQ right-hand sides, into nearbuf (point-major)
template <class T>
__global__ void __launch_bounds__(kLeafThreads) k_near_mr(LeafArgs A, const T *__restrict__ xs, T *__restrict__ nearbuf) {
    __shared__ __align__(16) float4 srcf[kMaxLeafMR * 2];          // FP32: hi, lo coordinates
    __shared__ __align__(16) Pt4d srcd[sizeof(T) == 8 ? kMaxLeafMR : 1];
    __shared__ T xsrc[kMaxLeafMR * kNQ];
    __shared__ T part[kLeafThreads * kNQ];
    const int z = blockIdx.x;
    const int Zg = (int)(A.offL + z);
    const int zs = A.box_start[Zg], m = A.box_end[Zg] - zs;
    const int T_ = kLeafThreads;
    const int S = m <= T_ ? max(1, T_ / m) : 1;
    const int ntg = m <= T_ ? 1 : (m + T_ - 1) / T_;   // at most 2 for m <= 256
    const int s = m <= T_ ? threadIdx.x / m : 0;
    const int i0 = m <= T_ ? threadIdx.x - s * m : threadIdx.x;
    const bool active = m <= T_ ? (s < S) : true;
    Acc<T> acc[2][kNQ];
    float4 th[2], tl[2];
    double tx[2], ty[2], tz[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int i = i0 + q * T_;
        const bool ok = active && q < ntg && i < m;
        if (sizeof(T) == 4) {
            th[q] = ok ? A.ploc[zs + i] : make_float4(0.f, 0.f, 0.f, 0.f);
            tl[q] = ok ? A.ploc_lo[zs + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            tx[q] = ok ? A.px[zs + i] : 0.0;
            ty[q] = ok ? A.py[zs + i] : 0.0;
            tz[q] = ok ? A.pz[zs + i] : 0.0;
        }
    }
    const float kap = (float)A.kappa;
    const int p1 = A.near_ptr[z + 1];
    int p = A.near_ptr[z];
    while (p < p1) {
        // stage near leaves [p, pe) together (up to kMaxLeafMR points)
        int pe = p, cnt = 0;
        while (pe < p1) {
            const int y = A.near_src[pe];
            const int n = A.box_end[A.offL + y] - A.box_start[A.offL + y];
            if (cnt + n > kMaxLeafMR && cnt > 0) break;
            cnt += n;
            ++pe;
        }
        __syncthreads();
        int base = 0;
        for (int pq = p; pq < pe; ++pq) {
            const int y = A.near_src[pq];
            const int ys = A.box_start[A.offL + y], n = A.box_end[A.offL + y] - ys;
            const int d = A.near_dir[pq];
            const float sx = (float)((d / 9 - 1) * A.hL), sy = (float)(((d / 3) % 3 - 1) * A.hL),
                        sz = (float)((d % 3 - 1) * A.hL);
            for (int j = threadIdx.x; j < n; j += T_) {
                if (sizeof(T) == 4) {
                    const float4 h = A.ploc[ys + j], l = A.ploc_lo[ys + j];
                    const float hx = h.x + sx, hy = h.y + sy, hz = h.z + sz;
                    srcf[2 * (base + j)] = make_float4(hx, hy, hz, 0.f);
                    srcf[2 * (base + j) + 1] = make_float4((h.x - (hx - sx)) + l.x, (h.y - (hy - sy)) + l.y,
                                                           (h.z - (hz - sz)) + l.z, 0.f);
                } else {
                    srcd[base + j] = make_pt4d(A.px[ys + j], A.py[ys + j], A.pz[ys + j], 0.0);
                }
            }
            for (int e = threadIdx.x; e < n * kNQ; e += T_) xsrc[base * kNQ + e] = xs[(int64_t)ys * kNQ + e];
            base += n;
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int i = i0 + q * T_;
                if (q >= ntg || i >= m) break;
                for (int j = s; j < cnt; j += S) {
                    T kij;
                    if (sizeof(T) == 4) {
                        const float4 sh = srcf[2 * j], sl = srcf[2 * j + 1];
                        const float dx = (th[q].x - sh.x) + (tl[q].x - sl.x);
                        const float dy = (th[q].y - sh.y) + (tl[q].y - sl.y);
                        const float dz = (th[q].z - sh.z) + (tl[q].z - sl.z);
                        kij = (T)kernel_fast(A.kind, kap, fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
                    } else {
                        const Pt4d sp = srcd[j];
                        const double dx = tx[q] - sp.x, dy = ty[q] - sp.y, dz = tz[q] - sp.z;
                        kij = (T)kernel_fast(A.kind, A.kappa, fma(dz, dz, fma(dy, dy, dx * dx)));
                    }
                    const T *xj = xsrc + j * kNQ;
#pragma unroll
                    for (int u = 0; u < kNQ; ++u) acc[q][u].add(kij * xj[u]);
                }
            }
        }
        p = pe;
    }
    __syncthreads();
    if (m <= T_) {
        if (active)
#pragma unroll
            for (int u = 0; u < kNQ; ++u) part[threadIdx.x * kNQ + u] = acc[0][u].get();
        __syncthreads();
        for (int e = threadIdx.x; e < m * kNQ; e += T_) {
            const int i = e / kNQ, u = e - i * kNQ;
            T v = 0;
            for (int g = 0; g < S; ++g) v += part[(g * m + i) * kNQ + u];
            nearbuf[(int64_t)(zs + i) * kNQ + u] = v;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = i0 + q * T_;
            if (q < ntg && i < m)
#pragma unroll
                for (int u = 0; u < kNQ; ++u) nearbuf[(int64_t)(zs + i) * kNQ + u] = acc[q][u].get();
        }
    }
}

// far field of one leaf for kNQ right-hand sides (TMA ring as k_leaf), plus the
// near field, written to columns q0 .. q0+nq-1 of y in the caller's order
template <class T>
__global__ void __launch_bounds__(kLeafThreads) k_leaf_mr(LeafArgs A, const T *__restrict__ U, const T *__restrict__ t,
                                                          const T *__restrict__ nearbuf, T *__restrict__ y, int64_t n,
                                                          int q0, int nq) {
    constexpr int W = Vec<T>::W;
    extern __shared__ __align__(128) unsigned char stage[];
    __shared__ __align__(8) uint64_t bars[kStages];
    __shared__ ChunkPlan P;
    __shared__ T red[kLeafThreads * W];
    const int z = blockIdx.x;
    const int Zg = (int)(A.offL + z);
    const int zs = A.box_start[Zg], m = A.box_end[Zg] - zs;
    const int ld = A.leaf_ld[z];
    const int nr = ld / W;                                  // <= kLeafThreads for leaves <= kMaxLeafMR
    const int cpc = kChunkBytes / (ld * (int)sizeof(T));
    const int L = A.L;
    if (threadIdx.x >= 1 && threadIdx.x <= L) {
        const int l = threadIdx.x;
        const int Ag = A.leaf_anc[(int64_t)(l - 1) * A.nleaf + z];
        const int RA = A.R[Ag];
        P.panel[l] = U + A.ubase[Ag] + (A.leaf_lp[z] - A.leaf_lp[A.leaf_lo[Ag]]) * RA;
        P.tA[l] = t + A.tbase[Ag] * kNQ;
        P.R[l] = RA;
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < kStages; ++q) mbar_init(&bars[q], 1);
        mbar_fence_init();
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
    int pl = 1;
    auto issue = [&](int k) {
        int c0, nc;
        chunk_of<T>(P, L, k, cpc, pl, c0, nc);
        const uint32_t bytes = (uint32_t)(nc * ld * (int)sizeof(T));
        uint64_t *bar = &bars[k % kStages];
        mbar_arrive_expect_tx(bar, bytes);
        bulk_copy_g2s(stage + (size_t)(k % kStages) * kChunkBytes,
                      static_cast<const T *>(P.panel[pl]) + (int64_t)c0 * ld, bytes, bar);
    };
    if (threadIdx.x == 0)
        for (int k = 0; k < min(kStages - 1, nchunks); ++k) issue(k);
    const int Gc = kLeafThreads / nr;
    const int g = threadIdx.x / nr;
    const int rv = threadIdx.x - g * nr;
    Acc<T> acc[W][kNQ];
    int cl_level = 1;
    for (int k = 0; k < nchunks; ++k) {
        const bool ok = mbar_wait(&bars[k % kStages], (uint32_t)((k / kStages) & 1));
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                *A.err = H3D_ERR_TIMEOUT;
                for (int j = k; j < min(k + kStages - 1, nchunks); ++j)
                    mbar_wait(&bars[j % kStages], (uint32_t)((j / kStages) & 1));
            }
            return;
        }
        if (threadIdx.x == 0 && k + kStages - 1 < nchunks) issue(k + kStages - 1);
        int c0, nc;
        chunk_of<T>(P, L, k, cpc, cl_level, c0, nc);
        const T *sm = reinterpret_cast<const T *>(stage + (size_t)(k % kStages) * kChunkBytes) + rv * W;
        const T *tA = static_cast<const T *>(P.tA[cl_level]) + (int64_t)c0 * kNQ;
        if (g < Gc) {
            int c = g;
            // four columns per compensated add
            for (; c + 3 * Gc < nc; c += 4 * Gc) {
                T part[W][kNQ];
#pragma unroll
                for (int e = 0; e < W; ++e)
#pragma unroll
                    for (int u = 0; u < kNQ; ++u) part[e][u] = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int cj = c + j * Gc;
                    T a[W];
                    Vec<T>::get(*reinterpret_cast<const typename Vec<T>::type *>(sm + cj * ld), a);
#pragma unroll
                    for (int u = 0; u < kNQ; u += W) {
                        T b[W];
                        Vec<T>::get(__ldg(reinterpret_cast<const typename Vec<T>::type *>(tA + (int64_t)cj * kNQ + u)), b);
#pragma unroll
                        for (int e = 0; e < W; ++e)
#pragma unroll
                            for (int f = 0; f < W; ++f) part[e][u + f] = fma(a[e], b[f], part[e][u + f]);
                    }
                }
#pragma unroll
                for (int e = 0; e < W; ++e)
#pragma unroll
                    for (int u = 0; u < kNQ; ++u) acc[e][u].add(part[e][u]);
            }
            for (; c < nc; c += Gc) {
                T a[W];
                Vec<T>::get(*reinterpret_cast<const typename Vec<T>::type *>(sm + c * ld), a);
#pragma unroll
                for (int u = 0; u < kNQ; u += W) {
                    T b[W];
                    Vec<T>::get(__ldg(reinterpret_cast<const typename Vec<T>::type *>(tA + (int64_t)c * kNQ + u)), b);
#pragma unroll
                    for (int e = 0; e < W; ++e)
#pragma unroll
                        for (int f = 0; f < W; ++f) acc[e][u + f].add(a[e] * b[f]);
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kNQ; ++u) {
        if (u < nq) {   // nq is uniform over the CTA
            if (g < Gc)
#pragma unroll
                for (int e = 0; e < W; ++e) red[g * ld + rv * W + e] = acc[e][u].get();
            __syncthreads();
            for (int i = threadIdx.x; i < m; i += kLeafThreads) {
                T v = 0;
                for (int q = 0; q < Gc; ++q) v += red[q * ld + i];
                y[(int64_t)(q0 + u) * n + A.perm[zs + i]] = v + nearbuf[(int64_t)(zs + i) * kNQ + u];
            }
            __syncthreads();
        }
    }
}

// ===========================================================================
// Wide blocks: kNQW = 32 right-hand sides per pass (nrhs > kNQ), FP32, leaves
// of up to kMaxLeafW points.  One thread owns one factor row / column and all
// 32 right-hand sides (compensated sums over groups of four products).
constexpr int kNQW = 32;
constexpr int kMaxLeafW = 128;

__global__ void k_permute_in_w(const float *__restrict__ x, int64_t n, int q0, int nq, const int *__restrict__ perm,
                               float *__restrict__ xs) {
    // thread per (point, rhs): coalesced writes of the point-major block
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * kNQW) return;
    const int64_t i = e / kNQW;
    const int q = (int)(e - i * kNQW);
    xs[e] = q < nq ? x[(int64_t)(q0 + q) * n + perm[i]] : 0.f;
}

// T_Y(c, :) = sum_r V_Y(r, c) x(r, :) on CUDA cores, one column per thread
__global__ void __launch_bounds__(kGatherThreads) k_gather_w(GatherArgs G, const float *__restrict__ V,
                                                             const float *__restrict__ xs, float *__restrict__ t,
                                                             float *__restrict__ partial) {
    constexpr int RC = 64;   // rows staged per chunk
    __shared__ __align__(16) float xsm[RC * kNQW];
    const int4 task = G.task[blockIdx.x];
    const int Y = task.x, r0 = task.y, r1 = task.z;
    const int nrows = r1 - r0;
    const int ld = G.ldv[Y], RvY = G.Rv[Y];
    const float *Vb = V + G.vbase[Y] + (int64_t)r0 * ld;
    const int64_t ys = (int64_t)G.box_start[Y] + r0;
    const bool direct = task.w != 0;
    const int64_t pb = G.pbase[blockIdx.x];
    const int64_t vc0 = G.vcol0[Y];
    for (int cb = 0; cb < RvY; cb += kGatherThreads) {
        const int c = cb + threadIdx.x;
        const bool act = c < RvY;
        Acc<float> acc[kNQW];
        for (int rc = 0; rc < nrows; rc += RC) {
            const int nr = min(RC, nrows - rc);
            __syncthreads();
            for (int e = threadIdx.x; e < nr * kNQW; e += kGatherThreads) xsm[e] = xs[(ys + rc) * kNQW + e];
            __syncthreads();
            if (act) {
                const float *p = Vb + (int64_t)rc * ld + c;
                int r = 0;
                for (; r + 4 <= nr; r += 4) {
                    const float a0 = __ldcs(p + (int64_t)r * ld), a1 = __ldcs(p + (int64_t)(r + 1) * ld),
                                a2 = __ldcs(p + (int64_t)(r + 2) * ld), a3 = __ldcs(p + (int64_t)(r + 3) * ld);
                    const float4 *x0 = reinterpret_cast<const float4 *>(xsm + r * kNQW);
#pragma unroll
                    for (int u = 0; u < kNQW / 4; ++u) {
                        const float4 b0 = x0[u], b1 = x0[u + kNQW / 4], b2 = x0[u + kNQW / 2], b3 = x0[u + 3 * kNQW / 4];
                        acc[4 * u + 0].add(a0 * b0.x + a1 * b1.x + a2 * b2.x + a3 * b3.x);
                        acc[4 * u + 1].add(a0 * b0.y + a1 * b1.y + a2 * b2.y + a3 * b3.y);
                        acc[4 * u + 2].add(a0 * b0.z + a1 * b1.z + a2 * b2.z + a3 * b3.z);
                        acc[4 * u + 3].add(a0 * b0.w + a1 * b1.w + a2 * b2.w + a3 * b3.w);
                    }
                }
                for (; r < nr; ++r) {
                    const float a = __ldcs(p + (int64_t)r * ld);
#pragma unroll
                    for (int u = 0; u < kNQW; ++u) acc[u].add(a * xsm[r * kNQW + u]);
                }
            }
        }
        if (act) {
            float *o = direct ? t + G.map_v[vc0 + c] * kNQW : partial + (pb + c) * kNQW;
#pragma unroll
            for (int u = 0; u < kNQW; u += 4)
                *reinterpret_cast<float4 *>(o + u) = make_float4(acc[u].get(), acc[u + 1].get(), acc[u + 2].get(),
                                                                 acc[u + 3].get());
        }
    }
}

__global__ void k_reduce_partials_w(SplitArgs S, const float *__restrict__ partial, float *__restrict__ t) {
    const int q = blockIdx.x;
    const int Y = S.box[q], nt = S.ntask[q], ld = S.ldv[Y], R = S.Rv[Y];
    const int64_t pb = S.pbase[q], vc0 = S.vcol0[Y];
    for (int e = threadIdx.x; e < R * kNQW; e += blockDim.x) {
        const int c = e / kNQW, j = e - c * kNQW;
        float v = 0.f;
        for (int k = 0; k < nt; ++k) v += partial[(pb + (int64_t)k * ld + c) * kNQW + j];
        t[S.map_v[vc0 + c] * kNQW + j] = v;
    }
}

// near field for 32 right-hand sides: one thread per (target, source group)
__global__ void __launch_bounds__(kLeafThreads) k_near_w(LeafArgs A, const float *__restrict__ xs,
                                                         float *__restrict__ nearbuf) {
    constexpr int CAP = 128;   // staged sources per pass
    __shared__ __align__(16) float4 srcf[CAP * 2];
    __shared__ __align__(16) float xsrc[CAP * kNQW];
    __shared__ float part[kLeafThreads * kNQW / 4];   // reduction in four slices of 8 right-hand sides
    for (int z = blockIdx.x; z < A.nleaf; z += gridDim.x) {
        const int Zg = (int)(A.offL + z);
        const int zs = A.box_start[Zg], m = A.box_end[Zg] - zs;
        const int T_ = kLeafThreads;
        const int S = max(1, T_ / m);          // m <= kMaxLeafW = T_
        const int s = threadIdx.x / m, i = threadIdx.x - s * m;
        const bool active = s < S;
        Acc<float> acc[kNQW];
        const float4 th = active ? A.ploc[zs + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 tl = active ? A.ploc_lo[zs + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float kap = (float)A.kappa;
        const int p1 = A.near_ptr[z + 1];
        int p = A.near_ptr[z];
        while (p < p1) {
            int pe = p, cnt = 0;
            while (pe < p1) {
                const int y = A.near_src[pe];
                const int nn = A.box_end[A.offL + y] - A.box_start[A.offL + y];
                if (cnt + nn > CAP && cnt > 0) break;
                cnt += nn;
                ++pe;
            }
            __syncthreads();
            int base = 0;
            for (int pq = p; pq < pe; ++pq) {
                const int y = A.near_src[pq];
                const int ys = A.box_start[A.offL + y], nn = A.box_end[A.offL + y] - ys;
                const int d = A.near_dir[pq];
                const float sx = (float)((d / 9 - 1) * A.hL), sy = (float)(((d / 3) % 3 - 1) * A.hL),
                            sz = (float)((d % 3 - 1) * A.hL);
                for (int j = threadIdx.x; j < nn; j += T_) {
                    const float4 h = A.ploc[ys + j], l = A.ploc_lo[ys + j];
                    const float hx = h.x + sx, hy = h.y + sy, hz = h.z + sz;
                    srcf[2 * (base + j)] = make_float4(hx, hy, hz, 0.f);
                    srcf[2 * (base + j) + 1] = make_float4((h.x - (hx - sx)) + l.x, (h.y - (hy - sy)) + l.y,
                                                           (h.z - (hz - sz)) + l.z, 0.f);
                }
                for (int e = threadIdx.x; e < nn * kNQW; e += T_) xsrc[base * kNQW + e] = xs[(int64_t)ys * kNQW + e];
                base += nn;
            }
            __syncthreads();
            if (active) {
                for (int j = s; j < cnt; j += S) {
                    const float4 sh = srcf[2 * j], sl = srcf[2 * j + 1];
                    const float dx = (th.x - sh.x) + (tl.x - sl.x);
                    const float dy = (th.y - sh.y) + (tl.y - sl.y);
                    const float dz = (th.z - sh.z) + (tl.z - sl.z);
                    const float kij = kernel_fast(A.kind, kap, fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
                    const float4 *xj = reinterpret_cast<const float4 *>(xsrc + j * kNQW);
#pragma unroll
                    for (int u = 0; u < kNQW / 4; ++u) {
                        const float4 b = xj[u];
                        acc[4 * u].add(kij * b.x);
                        acc[4 * u + 1].add(kij * b.y);
                        acc[4 * u + 2].add(kij * b.z);
                        acc[4 * u + 3].add(kij * b.w);
                    }
                }
            }
            p = pe;
        }
#pragma unroll
        for (int sl4 = 0; sl4 < 4; ++sl4) {
            __syncthreads();
            if (active)
#pragma unroll
                for (int u = 0; u < 8; ++u) part[threadIdx.x * 8 + u] = acc[sl4 * 8 + u].get();
            __syncthreads();
            for (int e = threadIdx.x; e < m * 8; e += T_) {
                const int ii = e / 8, u = e - ii * 8;
                float v = 0.f;
                for (int g = 0; g < S; ++g) v += part[(g * m + ii) * 8 + u];
                nearbuf[(int64_t)(zs + ii) * kNQW + sl4 * 8 + u] = v;
            }
        }
        __syncthreads();
    }
}

// far field for 32 right-hand sides: U panels through the TMA ring as k_leaf;
// one thread per (row, column group), all 32 right-hand sides
__global__ void __launch_bounds__(kLeafThreads) k_leaf_w(LeafArgs A, const float *__restrict__ U,
                                                         const float *__restrict__ t, const float *__restrict__ nearbuf,
                                                         float *__restrict__ y, int64_t n, int q0, int nq) {
    extern __shared__ __align__(128) unsigned char stage[];
    __shared__ __align__(8) uint64_t bars[kStages];
    __shared__ ChunkPlan P;
    __shared__ float red[kLeafThreads * 8];
    const int z = blockIdx.x;
    const int Zg = (int)(A.offL + z);
    const int zs = A.box_start[Zg], m = A.box_end[Zg] - zs;
    const int ld = A.leaf_ld[z];                            // <= kMaxLeafW
    const int cpc = kChunkBytes / (ld * (int)sizeof(float));
    const int L = A.L;
    if (threadIdx.x >= 1 && threadIdx.x <= L) {
        const int l = threadIdx.x;
        const int Ag = A.leaf_anc[(int64_t)(l - 1) * A.nleaf + z];
        const int RA = A.R[Ag];
        P.panel[l] = U + A.ubase[Ag] + (A.leaf_lp[z] - A.leaf_lp[A.leaf_lo[Ag]]) * RA;
        P.tA[l] = t + A.tbase[Ag] * kNQW;
        P.R[l] = RA;
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < kStages; ++q) mbar_init(&bars[q], 1);
        mbar_fence_init();
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
    int pl = 1;
    auto issue = [&](int k) {
        int c0, nc;
        chunk_of<float>(P, L, k, cpc, pl, c0, nc);
        const uint32_t bytes = (uint32_t)(nc * ld * (int)sizeof(float));
        uint64_t *bar = &bars[k % kStages];
        mbar_arrive_expect_tx(bar, bytes);
        bulk_copy_g2s(stage + (size_t)(k % kStages) * kChunkBytes,
                      static_cast<const float *>(P.panel[pl]) + (int64_t)c0 * ld, bytes, bar);
    };
    if (threadIdx.x == 0)
        for (int k = 0; k < min(kStages - 1, nchunks); ++k) issue(k);
    const int Gc = kLeafThreads / ld;
    const int g = threadIdx.x / ld, i = threadIdx.x - g * ld;
    Acc<float> acc[kNQW];
    int cl_level = 1;
    for (int k = 0; k < nchunks; ++k) {
        const bool ok = mbar_wait(&bars[k % kStages], (uint32_t)((k / kStages) & 1));
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                *A.err = H3D_ERR_TIMEOUT;
                for (int j = k; j < min(k + kStages - 1, nchunks); ++j)
                    mbar_wait(&bars[j % kStages], (uint32_t)((j / kStages) & 1));
            }
            return;
        }
        if (threadIdx.x == 0 && k + kStages - 1 < nchunks) issue(k + kStages - 1);
        int c0, nc;
        chunk_of<float>(P, L, k, cpc, cl_level, c0, nc);
        const float *sm = reinterpret_cast<const float *>(stage + (size_t)(k % kStages) * kChunkBytes) + i;
        const float *tA = static_cast<const float *>(P.tA[cl_level]) + (int64_t)c0 * kNQW;
        if (g < Gc) {
            int c = g;
            for (; c + 3 * Gc < nc; c += 4 * Gc) {
                const float a0 = sm[c * ld], a1 = sm[(c + Gc) * ld], a2 = sm[(c + 2 * Gc) * ld],
                            a3 = sm[(c + 3 * Gc) * ld];
                const float4 *b0 = reinterpret_cast<const float4 *>(tA + (int64_t)c * kNQW);
                const float4 *b1 = reinterpret_cast<const float4 *>(tA + (int64_t)(c + Gc) * kNQW);
                const float4 *b2 = reinterpret_cast<const float4 *>(tA + (int64_t)(c + 2 * Gc) * kNQW);
                const float4 *b3 = reinterpret_cast<const float4 *>(tA + (int64_t)(c + 3 * Gc) * kNQW);
#pragma unroll
                for (int u = 0; u < kNQW / 4; ++u) {
                    const float4 v0 = __ldg(b0 + u), v1 = __ldg(b1 + u), v2 = __ldg(b2 + u), v3 = __ldg(b3 + u);
                    acc[4 * u].add(a0 * v0.x + a1 * v1.x + a2 * v2.x + a3 * v3.x);
                    acc[4 * u + 1].add(a0 * v0.y + a1 * v1.y + a2 * v2.y + a3 * v3.y);
                    acc[4 * u + 2].add(a0 * v0.z + a1 * v1.z + a2 * v2.z + a3 * v3.z);
                    acc[4 * u + 3].add(a0 * v0.w + a1 * v1.w + a2 * v2.w + a3 * v3.w);
                }
            }
            for (; c < nc; c += Gc) {
                const float a = sm[c * ld];
                const float4 *b = reinterpret_cast<const float4 *>(tA + (int64_t)c * kNQW);
#pragma unroll
                for (int u = 0; u < kNQW / 4; ++u) {
                    const float4 v = __ldg(b + u);
                    acc[4 * u].add(a * v.x);
                    acc[4 * u + 1].add(a * v.y);
                    acc[4 * u + 2].add(a * v.z);
                    acc[4 * u + 3].add(a * v.w);
                }
            }
        }
    }
    // reduce over column groups in four slices of 8 right-hand sides
#pragma unroll
    for (int sl4 = 0; sl4 < 4; ++sl4) {
        __syncthreads();
        if (g < Gc)
#pragma unroll
            for (int u = 0; u < 8; ++u) red[(g * ld + i) * 8 + u] = acc[sl4 * 8 + u].get();
        __syncthreads();
        for (int e = threadIdx.x; e < m * 8; e += kLeafThreads) {
            const int ii = e / 8, u = e - ii * 8, q = sl4 * 8 + u;
            if (q >= nq) continue;
            float v = 0.f;
            for (int gg = 0; gg < Gc; ++gg) v += red[(gg * ld + ii) * 8 + u];
            y[(int64_t)(q0 + q) * n + A.perm[zs + ii]] = v + nearbuf[(int64_t)(zs + ii) * kNQW + q];
        }
    }
}

// ===========================================================================
// Source-side gather of 32 right-hand sides on the tensor cores (tcgen05,
// kind::tf32, 3xTF32 split precision):
//   T_Y(c, q) = sum_r V_Y(r, c) x(r, q)  as  D[M = c][N = q] += A[M][K = r] B[K][N].
// A work item is one gather task (source box, row range) and a tile of 128
// columns.  Per K step of 8 rows every thread loads V and x, splits each value
// into tf32 hi + lo (the tensor core truncates FP32 operands to tf32, so both
// parts are rounded here) and writes them into K-major core-matrix layout (8 rows
// x 16 bytes per core matrix; LBO = 128 B along K, SBO = 256 B along M or N) in one
// of two shared-memory buffers; one thread issues the MMAs and commits them to the
// buffer's mbarrier, which the threads wait on (bounded) before refilling it.
// Accumulation: the tensor core's FP32 accumulation is biased (its error grows
// about one ulp per accumulated MMA), so the main products hi*hi go to one of two
// TMEM accumulators that is restarted every kTcGroup K steps and drained into a
// compensated FP32 sum in registers while the other one is filled; the small
// corrections hi*lo + lo*hi (2^-11 of the main term) accumulate in a third TMEM
// accumulator over the whole item.  The CTAs are persistent and keep their TMEM
// allocation for the whole launch.
constexpr int kTcThreads = 128;
constexpr int kTcGroup = 4;                           // K steps per drained accumulator
constexpr int kTcAOp = 4096;                          // one A operand: 128 rows x 8 k, tf32
constexpr int kTcBOp = 1024;                          // one B operand: 32 columns x 8 k
constexpr int kTcBuf = 2 * kTcAOp + 2 * kTcBOp;       // hi and lo of A and B
constexpr size_t kTcDynSmem = 2 * (size_t)kTcBuf + 128;
constexpr int kTcCtasPerSm = 3;
constexpr int kTcCols = 128;

__global__ void __launch_bounds__(kTcThreads) k_gather_tc(GatherArgs G, const int2 *__restrict__ items, int nitems,
                                                          const float *__restrict__ V, const float *__restrict__ xs,
                                                          float *__restrict__ t, float *__restrict__ partial,
                                                          int *err) {
    extern __shared__ unsigned char dsm_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    unsigned char *dsm = dsm_raw + ((128 - (smem_addr(dsm_raw) & 127)) & 127);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tmem_alloc(&tmem_base, 128);   // main[0], main[1], corrections, unused
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t tlane = (uint32_t)(warp << 5) << 16;   // this warp's TMEM lanes
    const uint32_t idesc = umma_idesc_tf32(128, kNQW);
    uint32_t issued[2] = {0u, 0u}, waited[2] = {0u, 0u};
    int step = 0;
    bool failed = false;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 w = items[it];
        const int4 task = G.task[w.x];
        const int Y = task.x, r0 = task.y, r1 = task.z;
        const int ld = G.ldv[Y], RvY = G.Rv[Y];
        const int c_lo = w.y * kTcCols;
        const int ncols = min(kTcCols, RvY - c_lo);
        const float *Vb = V + G.vbase[Y] + (int64_t)r0 * ld + c_lo;
        const int64_t xrow0 = (int64_t)G.box_start[Y] + r0;
        const int nrows = r1 - r0;
        const int nsteps = (nrows + 7) >> 3;
        const int ngroups = (nsteps + kTcGroup - 1) / kTcGroup;
        Acc<float> acc[kNQW];
        auto drain = [&](int grp) {   // add main accumulator of group grp into the register sums
            float v[32];
            tmem_ld32(tmem + tlane + 32u * (uint32_t)(grp & 1), v);
#pragma unroll
            for (int q = 0; q < kNQW; ++q) acc[q].add(v[q]);
        };
        for (int s = 0; s < nsteps; ++s, ++step) {
            const int b = step & 1;
            unsigned char *buf = dsm + b * kTcBuf;
            if (issued[b] != waited[b]) {   // the MMAs that read this buffer must be done
                const bool ok = mbar_wait(&mbar[b], waited[b] & 1u);
                ++waited[b];
                if (__syncthreads_or(!ok)) { failed = true; break; }
                tc_fence_after();
            }
            const int grp = s / kTcGroup;
            // the accumulator this group reuses held group grp-2, complete by now
            if (s % kTcGroup == 0 && grp >= 2) drain(grp - 2);
            const int rk = s << 3;
            {   // A: 8 rows x 128 columns of V, one column per thread
                const bool colok = tid < ncols;
                float hi[8], lo[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int r = rk + k;
                    const float v = (colok && r < nrows) ? __ldcs(Vb + (int64_t)r * ld + tid) : 0.f;
                    split_tf32(v, hi[k], lo[k]);
                }
                unsigned char *ah = buf + ((tid >> 3) << 8) + ((tid & 7) << 4);
                *reinterpret_cast<float4 *>(ah) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<float4 *>(ah + 128) = make_float4(hi[4], hi[5], hi[6], hi[7]);
                *reinterpret_cast<float4 *>(ah + kTcAOp) = make_float4(lo[0], lo[1], lo[2], lo[3]);
                *reinterpret_cast<float4 *>(ah + kTcAOp + 128) = make_float4(lo[4], lo[5], lo[6], lo[7]);
            }
            {   // B: 8 rows x 32 right-hand sides of x, two values per thread
                const int n = tid & 31, k0 = (tid >> 5) << 1;
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const int k = k0 + kk, r = rk + k;
                    const float v = r < nrows ? xs[(xrow0 + r) * kNQW + n] : 0.f;
                    float h, l;
                    split_tf32(v, h, l);
                    const int off = ((n >> 3) << 8) + ((k >> 2) << 7) + ((n & 7) << 4) + ((k & 3) << 2);
                    *reinterpret_cast<float *>(buf + 2 * kTcAOp + off) = h;
                    *reinterpret_cast<float *>(buf + 2 * kTcAOp + kTcBOp + off) = l;
                }
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) {
                const uint32_t abase = smem_addr(buf), bbase = abase + 2 * kTcAOp;
                const uint64_t ahd = umma_desc(abase, 128, 256), ald = umma_desc(abase + kTcAOp, 128, 256);
                const uint64_t bh = umma_desc(bbase, 128, 256), bl = umma_desc(bbase + kTcBOp, 128, 256);
                umma_tf32(tmem + 32u * (uint32_t)(grp & 1), ahd, bh, idesc, s % kTcGroup ? 1u : 0u);
                umma_tf32(tmem + 64u, ahd, bl, idesc, s > 0 ? 1u : 0u);
                umma_tf32(tmem + 64u, ald, bh, idesc, 1u);
                umma_commit(&mbar[b]);
            }
            ++issued[b];
        }
        if (failed) break;
        bool ok = true;
        for (int bb = 0; bb < 2; ++bb)
            while (waited[bb] != issued[bb]) {
                ok = mbar_wait(&mbar[bb], waited[bb] & 1u) && ok;
                ++waited[bb];
            }
        if (__syncthreads_or(!ok)) { failed = true; break; }
        tc_fence_after();
        if (ngroups >= 2) drain(ngroups - 2);
        drain(ngroups - 1);
        {
            float v[32];
            tmem_ld32(tmem + tlane + 64u, v);
#pragma unroll
            for (int q = 0; q < kNQW; ++q) acc[q].add(v[q]);
        }
        const int m = (warp << 5) + lane;
        if (m < ncols) {
            const int c = c_lo + m;
            float *o = task.w ? t + G.map_v[G.vcol0[Y] + c] * kNQW : partial + (G.pbase[w.x] + c) * kNQW;
#pragma unroll
            for (int q = 0; q < kNQW; q += 4)
                *reinterpret_cast<float4 *>(o + q) =
                    make_float4(acc[q].get(), acc[q + 1].get(), acc[q + 2].get(), acc[q + 3].get());
        }
        tc_fence_before();
        __syncthreads();   // accumulators read before the next item overwrites them
        tc_fence_after();
    }
    if (failed && tid == 0) *err = H3D_ERR_TIMEOUT;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

// Far field of one leaf for 32 right-hand sides on the tensor cores:
//   y(rows, q) = sum over levels of U_panel(rows, c) t_A(c, q)
// as D[M = 128 rows (the leaf's rows, the rest zero)][N = 32] += A[M][K = c] B[K][N].
// The U panels arrive through the same TMA ring as in k_leaf; per K step of 8
// columns the threads split U (transposed into K-major) and t into tf32 hi + lo
// operands; accumulation as in k_gather_tc (drained main accumulators, one
// correction accumulator).  Then far + near in the caller's order.
constexpr size_t kLeafTcDynSmem = kLeafDynSmem + 2 * (size_t)kTcBuf + 128;

__global__ void __launch_bounds__(kTcThreads) k_leaf_tc(LeafArgs A, const float *__restrict__ U,
                                                        const float *__restrict__ t, const float *__restrict__ nearbuf,
                                                        float *__restrict__ y, int64_t n, int q0, int nq) {
    extern __shared__ __align__(128) unsigned char stage[];   // TMA ring, then the operand buffers
    __shared__ __align__(8) uint64_t bars[kStages];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ ChunkPlan P;
    __shared__ uint32_t tmem_base;
    unsigned char *ops_raw = stage + kLeafDynSmem;
    unsigned char *ops = ops_raw + ((128 - (smem_addr(ops_raw) & 127)) & 127);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int z = blockIdx.x;
    const int Zg = (int)(A.offL + z);
    const int zs = A.box_start[Zg], m = A.box_end[Zg] - zs;
    const int ld = A.leaf_ld[z];                               // <= kMaxLeafW = 128
    const int cpc = kChunkBytes / (ld * (int)sizeof(float));
    const int L = A.L;
    if (warp == 0) tmem_alloc(&tmem_base, 128);
    if (tid >= 1 && tid <= L) {
        const int l = tid;
        const int Ag = A.leaf_anc[(int64_t)(l - 1) * A.nleaf + z];
        const int RA = A.R[Ag];
        P.panel[l] = U + A.ubase[Ag] + (A.leaf_lp[z] - A.leaf_lp[A.leaf_lo[Ag]]) * RA;
        P.tA[l] = t + A.tbase[Ag] * kNQW;
        P.R[l] = RA;
    }
    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) mbar_init(&bars[q], 1);
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_fence_init();
    }
    // rows >= ld of the A operands stay zero
    for (int e = tid; e < 2 * kTcBuf / 16; e += kTcThreads)
        reinterpret_cast<float4 *>(ops)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        int acc = 0;
        for (int l = 1; l <= L; ++l) {
            P.first[l] = acc;
            acc += (P.R[l] + cpc - 1) / cpc;
        }
        P.first[L + 1] = acc;
    }
    __syncthreads();
    const uint32_t tmem = tmem_base;
    const uint32_t tlane = (uint32_t)(warp << 5) << 16;
    const uint32_t idesc = umma_idesc_tf32(128, kNQW);
    const int nchunks = P.first[L + 1];
    int pl = 1;
    auto issue = [&](int k) {
        int c0, nc;
        chunk_of<float>(P, L, k, cpc, pl, c0, nc);
        const uint32_t bytes = (uint32_t)(nc * ld * (int)sizeof(float));
        uint64_t *bar = &bars[k % kStages];
        mbar_arrive_expect_tx(bar, bytes);
        bulk_copy_g2s(stage + (size_t)(k % kStages) * kChunkBytes,
                      static_cast<const float *>(P.panel[pl]) + (int64_t)c0 * ld, bytes, bar);
    };
    if (tid == 0)
        for (int k = 0; k < min(kStages - 1, nchunks); ++k) issue(k);
    Acc<float> acc[kNQW];
    auto drain = [&](int grp) {
        float v[32];
        tmem_ld32(tmem + tlane + 32u * (uint32_t)(grp & 1), v);
#pragma unroll
        for (int q = 0; q < kNQW; ++q) acc[q].add(v[q]);
    };
    uint32_t issued[2] = {0u, 0u}, waited[2] = {0u, 0u};
    int s = 0, cl_level = 1;
    bool failed = false;
    for (int k = 0; k < nchunks && !failed; ++k) {
        const bool okc = mbar_wait(&bars[k % kStages], (uint32_t)((k / kStages) & 1));
        if (__syncthreads_or(!okc)) { failed = true; break; }
        if (tid == 0 && k + kStages - 1 < nchunks) issue(k + kStages - 1);
        int c0, nc;
        chunk_of<float>(P, L, k, cpc, cl_level, c0, nc);
        const float *sm = reinterpret_cast<const float *>(stage + (size_t)(k % kStages) * kChunkBytes);
        const float *tA = static_cast<const float *>(P.tA[cl_level]) + (int64_t)c0 * kNQW;
        const int nks = (nc + 7) >> 3;
        for (int ks = 0; ks < nks; ++ks, ++s) {
            const int b = s & 1;
            unsigned char *buf = ops + b * kTcBuf;
            if (issued[b] != waited[b]) {
                const bool ok = mbar_wait(&mbar[b], waited[b] & 1u);
                ++waited[b];
                if (__syncthreads_or(!ok)) { failed = true; break; }
                tc_fence_after();
            }
            const int grp = s / kTcGroup;
            if (s % kTcGroup == 0 && grp >= 2) drain(grp - 2);
            const int cb = ks << 3;
            if (tid < ld) {   // A: row tid, 8 columns
                float hi[8], lo[8];
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const int c = cb + kk;
                    split_tf32(c < nc ? sm[c * ld + tid] : 0.f, hi[kk], lo[kk]);
                }
                unsigned char *ah = buf + ((tid >> 3) << 8) + ((tid & 7) << 4);
                *reinterpret_cast<float4 *>(ah) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<float4 *>(ah + 128) = make_float4(hi[4], hi[5], hi[6], hi[7]);
                *reinterpret_cast<float4 *>(ah + kTcAOp) = make_float4(lo[0], lo[1], lo[2], lo[3]);
                *reinterpret_cast<float4 *>(ah + kTcAOp + 128) = make_float4(lo[4], lo[5], lo[6], lo[7]);
            }
            {   // B: 8 columns x 32 right-hand sides of t, two values per thread
                const int nn = tid & 31, k0 = (tid >> 5) << 1;
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const int kq = k0 + kk, c = cb + kq;
                    const float v = c < nc ? __ldg(tA + (int64_t)c * kNQW + nn) : 0.f;
                    float h, l;
                    split_tf32(v, h, l);
                    const int off = ((nn >> 3) << 8) + ((kq >> 2) << 7) + ((nn & 7) << 4) + ((kq & 3) << 2);
                    *reinterpret_cast<float *>(buf + 2 * kTcAOp + off) = h;
                    *reinterpret_cast<float *>(buf + 2 * kTcAOp + kTcBOp + off) = l;
                }
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) {
                const uint32_t abase = smem_addr(buf), bbase = abase + 2 * kTcAOp;
                const uint64_t ahd = umma_desc(abase, 128, 256), ald = umma_desc(abase + kTcAOp, 128, 256);
                const uint64_t bh = umma_desc(bbase, 128, 256), bl = umma_desc(bbase + kTcBOp, 128, 256);
                umma_tf32(tmem + 32u * (uint32_t)(grp & 1), ahd, bh, idesc, s % kTcGroup ? 1u : 0u);
                umma_tf32(tmem + 64u, ahd, bl, idesc, s > 0 ? 1u : 0u);
                umma_tf32(tmem + 64u, ald, bh, idesc, 1u);
                umma_commit(&mbar[b]);
            }
            ++issued[b];
        }
    }
    if (!failed) {
        bool ok = true;
        for (int bb = 0; bb < 2; ++bb)
            while (waited[bb] != issued[bb]) {
                ok = mbar_wait(&mbar[bb], waited[bb] & 1u) && ok;
                ++waited[bb];
            }
        failed = __syncthreads_or(!ok);
    }
    if (!failed) {
        tc_fence_after();
        if (s > 0) {
            const int ngroups = (s + kTcGroup - 1) / kTcGroup;
            if (ngroups >= 2) drain(ngroups - 2);
            drain(ngroups - 1);
            float v[32];
            tmem_ld32(tmem + tlane + 64u, v);
#pragma unroll
            for (int q = 0; q < kNQW; ++q) acc[q].add(v[q]);
        }
        const int i = tid;
        if (i < m) {
            const int64_t o = A.perm[zs + i];
#pragma unroll
            for (int q = 0; q < kNQW; ++q)
                if (q < nq) y[(int64_t)(q0 + q) * n + o] = acc[q].get() + nearbuf[(int64_t)(zs + i) * kNQW + q];
        }
    } else if (tid == 0) {
        *A.err = H3D_ERR_TIMEOUT;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

unsigned gridn(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

LeafArgs leaf_args(const Handle &h) {
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

// transpose reduce work list (host-built)
struct TPlan {
    int n = 0;
    int *box = nullptr, *level = nullptr;
};

template <class T>
void matvec_one(Handle &h, const T *x, T *y, bool transpose, cudaStream_t s, cudaEvent_t *ev) {
    const int64_t n = h.N;
    T *xs = (T *)h.xs, *t = (T *)h.t;
    if (ev) H3D_CUDA(cudaEventRecord(ev[0], s));
    k_permute_in<T><<<gridn(n, 256), 256, 0, s>>>(x, h.perm, n, xs);
    if (ev) H3D_CUDA(cudaEventRecord(ev[1], s));
    LeafArgs A = leaf_args(h);
    T *nearbuf = (T *)h.nearbuf;
    // near field on the side stream, overlapping the factor streams
    H3D_CUDA(cudaEventRecord(h.ev_fork, s));
    H3D_CUDA(cudaStreamWaitEvent(h.side_stream, h.ev_fork, 0));
    // FP32: a small persistent grid that hides under the gather; FP64 (whose near
    // field is bound by the FP64 pipe, not hidden by anything): every leaf at once
    const int near_grid = sizeof(T) == 4 ? std::min(h.nleaf, kNearCtasPerSm * num_sms()) : h.nleaf;
    k_near<T><<<near_grid, kLeafThreads, 0, h.side_stream>>>(A, xs, nearbuf);
    H3D_CUDA(cudaEventRecord(h.ev_join, h.side_stream));
    if (!transpose) {
        if (h.ngtask > 0) {
            GatherArgs G{h.gtask, h.gtask_pbase, h.box_start, h.Rv, h.ldv, h.vbase, h.vcol0, h.map_v};
            k_gather<T><<<h.ngtask, kGatherThreads, 0, s>>>(G, (const T *)h.V, xs, t, (T *)h.partial);
        }
        if (ev) H3D_CUDA(cudaEventRecord(ev[2], s));
        if (h.nsplit > 0) {
            SplitArgs S{h.split_box, h.split_ntask, h.split_pbase, h.Rv, h.ldv, h.vcol0, h.map_v};
            k_reduce_partials<T><<<h.nsplit, 256, 0, s>>>(S, (const T *)h.partial, t);
        }
        H3D_CUDA(cudaStreamWaitEvent(s, h.ev_join, 0));
        if (ev) H3D_CUDA(cudaEventRecord(ev[3], s));
        k_leaf<T><<<h.nleaf, kLeafThreads, kLeafDynSmem, s>>>(A, (const T *)h.U, t, nearbuf, y);
        if (ev) H3D_CUDA(cudaEventRecord(ev[4], s));
    } else {
        if (h.nblk > 0) {
            k_leafT_gather<T><<<h.nleaf, kLeafThreads, 0, s>>>(A, (const T *)h.U, xs, t, (T *)h.tpartial);
            if (h.nsplit_T > 0) {
                ReduceTArgs R{h.tsplit_box, h.tsplit_level, h.R, h.box_leaf_lo, h.box_leaf_hi, h.tbase, h.tp_base,
                              h.nleaf};
                k_reduceT<T><<<h.nsplit_T, 256, 0, s>>>(R, (const T *)h.tpartial, t);
            }
        }
        H3D_CUDA(cudaStreamWaitEvent(s, h.ev_join, 0));
        k_leafT<T><<<h.nleaf, kLeafThreads, 0, s>>>(A, (const T *)h.V, t, nearbuf, y);
    }
    H3D_LAUNCH_CHECK();
}

void matvec_wide(Handle &h, const float *x, float *y, int q0, int nq, cudaStream_t s, cudaEvent_t *ev) {
    const int64_t n = h.N;
    float *xs = (float *)h.xs_w, *t = (float *)h.t_w, *nearbuf = (float *)h.nearbuf_w;
    if (ev) H3D_CUDA(cudaEventRecord(ev[0], s));
    k_permute_in_w<<<gridn(n * kNQW, 256), 256, 0, s>>>(x, n, q0, nq, h.perm, xs);
    if (ev) H3D_CUDA(cudaEventRecord(ev[1], s));
    LeafArgs A = leaf_args(h);
    H3D_CUDA(cudaEventRecord(h.ev_fork, s));
    H3D_CUDA(cudaStreamWaitEvent(h.side_stream, h.ev_fork, 0));
    k_near_w<<<std::min(h.nleaf, 2 * kNearCtasPerSm * num_sms()), kLeafThreads, 0, h.side_stream>>>(A, xs, nearbuf);
    H3D_CUDA(cudaEventRecord(h.ev_join, h.side_stream));
    if (h.ntc_items > 0) {
        GatherArgs G{h.gtask, h.gtask_pbase, h.box_start, h.Rv, h.ldv, h.vbase, h.vcol0, h.map_v};
        const int grid = std::min(h.ntc_items, kTcCtasPerSm * num_sms());
        k_gather_tc<<<grid, kTcThreads, kTcDynSmem, s>>>(G, h.tc_items, h.ntc_items, (const float *)h.V, xs, t,
                                                         (float *)h.partial_w, h.d_async_err);
    }
    if (ev) H3D_CUDA(cudaEventRecord(ev[2], s));
    if (h.nsplit > 0) {
        SplitArgs S{h.split_box, h.split_ntask, h.split_pbase, h.Rv, h.ldv, h.vcol0, h.map_v};
        k_reduce_partials_w<<<h.nsplit, 256, 0, s>>>(S, (const float *)h.partial_w, t);
    }
    H3D_CUDA(cudaStreamWaitEvent(s, h.ev_join, 0));
    if (ev) H3D_CUDA(cudaEventRecord(ev[3], s));
    k_leaf_tc<<<h.nleaf, kTcThreads, kLeafTcDynSmem, s>>>(A, (const float *)h.U, t, nearbuf, y, n, q0, nq);
    if (ev) H3D_CUDA(cudaEventRecord(ev[4], s));
    H3D_LAUNCH_CHECK();
}

// scratch of the 32-column path, allocated by the first product that needs it
void ensure_wide_scratch(Handle &h, cudaStream_t s) {
    if (h.xs_w) return;
    H3D_CUDA(cudaStreamSynchronize(s));
    const size_t es = sizeof(float);
    h.xs_w = h.mem.alloc((size_t)std::max<int64_t>(h.N, 4) * kNQW * es);
    h.nearbuf_w = h.mem.alloc((size_t)std::max<int64_t>(h.N, 4) * kNQW * es);
    h.t_w = h.mem.alloc((size_t)std::max<int64_t>(h.sum_rank, 4) * kNQW * es);
    h.partial_w = h.mem.alloc((size_t)std::max<int64_t>(h.partial_elems, 4) * kNQW * es);
}

bool use_wide(const Handle &h, int nrhs, bool transpose) {
    return nrhs > kNQ && !transpose && h.prec == H3D_FP32 && h.leaf_size <= kMaxLeafW;
}

template <class T>
void matvec_mr(Handle &h, const T *x, T *y, int q0, int nq, cudaStream_t s, cudaEvent_t *ev) {
    const int64_t n = h.N;
    T *xs = (T *)h.xs_mr, *t = (T *)h.t_mr, *nearbuf = (T *)h.nearbuf_mr;
    if (ev) H3D_CUDA(cudaEventRecord(ev[0], s));
    k_permute_in_mr<T><<<gridn(n, 256), 256, 0, s>>>(x, n, q0, nq, h.perm, xs);
    if (ev) H3D_CUDA(cudaEventRecord(ev[1], s));
    LeafArgs A = leaf_args(h);
    H3D_CUDA(cudaEventRecord(h.ev_fork, s));
    H3D_CUDA(cudaStreamWaitEvent(h.side_stream, h.ev_fork, 0));
    k_near_mr<T><<<h.nleaf, kLeafThreads, 0, h.side_stream>>>(A, xs, nearbuf);
    H3D_CUDA(cudaEventRecord(h.ev_join, h.side_stream));
    if (h.ngtask > 0) {
        GatherArgs G{h.gtask, h.gtask_pbase, h.box_start, h.Rv, h.ldv, h.vbase, h.vcol0, h.map_v};
        k_gather_mr<T><<<h.ngtask, kGatherThreads, 0, s>>>(G, (const T *)h.V, xs, t, (T *)h.partial_mr);
    }
    if (ev) H3D_CUDA(cudaEventRecord(ev[2], s));
    if (h.nsplit > 0) {
        SplitArgs S{h.split_box, h.split_ntask, h.split_pbase, h.Rv, h.ldv, h.vcol0, h.map_v};
        k_reduce_partials_mr<T><<<h.nsplit, 256, 0, s>>>(S, (const T *)h.partial_mr, t);
    }
    H3D_CUDA(cudaStreamWaitEvent(s, h.ev_join, 0));
    if (ev) H3D_CUDA(cudaEventRecord(ev[3], s));
    k_leaf_mr<T><<<h.nleaf, kLeafThreads, kLeafDynSmem, s>>>(A, (const T *)h.U, t, nearbuf, y, n, q0, nq);
    if (ev) H3D_CUDA(cudaEventRecord(ev[4], s));
    H3D_LAUNCH_CHECK();
}

}  // namespace

void build_matvec_plan(Handle &h, cudaStream_t s, Arena &tmp) {
    (void)tmp;
    H3D_CUDA(cudaFuncSetAttribute(k_leaf<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeafDynSmem));
    H3D_CUDA(cudaFuncSetAttribute(k_leaf<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeafDynSmem));
    H3D_CUDA(cudaFuncSetAttribute(k_leaf_mr<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeafDynSmem));
    H3D_CUDA(cudaFuncSetAttribute(k_leaf_mr<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeafDynSmem));
    H3D_CUDA(cudaFuncSetAttribute(k_leaf_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeafDynSmem));
    H3D_CUDA(cudaFuncSetAttribute(k_gather_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcDynSmem));
    H3D_CUDA(cudaFuncSetAttribute(k_leaf_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeafTcDynSmem));
    const int64_t nboxes = h.n_boxes;
    const size_t es = h.elem();
    std::vector<int> Rv(nboxes), ldv(nboxes), bs(nboxes), be(nboxes), R(nboxes), llo(nboxes), lhi(nboxes);
    H3D_CUDA(cudaMemcpyAsync(Rv.data(), h.Rv, nboxes * sizeof(int), cudaMemcpyDeviceToHost, s));
    H3D_CUDA(cudaMemcpyAsync(ldv.data(), h.ldv, nboxes * sizeof(int), cudaMemcpyDeviceToHost, s));
    H3D_CUDA(cudaMemcpyAsync(bs.data(), h.box_start, nboxes * sizeof(int), cudaMemcpyDeviceToHost, s));
    H3D_CUDA(cudaMemcpyAsync(be.data(), h.box_end, nboxes * sizeof(int), cudaMemcpyDeviceToHost, s));
    H3D_CUDA(cudaMemcpyAsync(R.data(), h.R, nboxes * sizeof(int), cudaMemcpyDeviceToHost, s));
    H3D_CUDA(cudaMemcpyAsync(llo.data(), h.box_leaf_lo, nboxes * sizeof(int), cudaMemcpyDeviceToHost, s));
    H3D_CUDA(cudaMemcpyAsync(lhi.data(), h.box_leaf_hi, nboxes * sizeof(int), cudaMemcpyDeviceToHost, s));
    H3D_CUDA(cudaStreamSynchronize(s));

    // gather tasks: coarse levels first (they are the longest)
    std::vector<int4> tasks;
    std::vector<int64_t> pbase;
    std::vector<int> sbox, stask0, sntask;
    std::vector<int64_t> spbase;
    int64_t pel = 0;
    for (int64_t g = 0; g < nboxes; ++g) {
        if (Rv[g] == 0) continue;
        const int n = be[g] - bs[g];
        int rows = (int)std::max<int64_t>(1, kTaskElems / std::max(1, ldv[g]));
        rows = std::min(rows, kTaskMaxRows);
        int nt = (n + rows - 1) / rows;
        if (nt == 2 && n <= kTaskMaxRows && (int64_t)n * ldv[g] <= 2 * kTaskElems) nt = 1;
        if (nt == 1) {
            tasks.push_back(make_int4((int)g, 0, n, 1));
            pbase.push_back(-1);
        } else {
            const int per = (n + nt - 1) / nt;
            sbox.push_back((int)g);
            stask0.push_back((int)tasks.size());
            sntask.push_back(nt);
            spbase.push_back(pel);
            for (int k = 0; k < nt; ++k) {
                tasks.push_back(make_int4((int)g, k * per, std::min(n, (k + 1) * per), 0));
                pbase.push_back(pel + (int64_t)k * ldv[g]);
            }
            pel += (int64_t)nt * ldv[g];
        }
    }
    h.ngtask = (int)tasks.size();
    h.gtask = h.mem.get<int4>(std::max<size_t>(tasks.size(), 1));
    h.gtask_pbase = h.mem.get<int64_t>(std::max<size_t>(pbase.size(), 1));
    if (!tasks.empty()) {
        H3D_CUDA(cudaMemcpyAsync(h.gtask, tasks.data(), tasks.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
        H3D_CUDA(cudaMemcpyAsync(h.gtask_pbase, pbase.data(), pbase.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    }
    // tensor-core gather work items: (task, block of kTcCols columns)
    {
        std::vector<int2> items;
        for (size_t q = 0; q < tasks.size(); ++q) {
            const int nb = (Rv[tasks[q].x] + kTcCols - 1) / kTcCols;
            for (int cb = 0; cb < nb; ++cb) items.push_back(make_int2((int)q, cb));
        }
        h.ntc_items = (int)items.size();
        h.tc_items = h.mem.get<int2>(std::max<size_t>(items.size(), 1));
        if (!items.empty())
            H3D_CUDA(cudaMemcpyAsync(h.tc_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    }
    h.nsplit = (int)sbox.size();
    h.split_box = h.mem.get<int>(std::max<size_t>(sbox.size(), 1));
    h.split_task0 = h.mem.get<int>(std::max<size_t>(sbox.size(), 1));
    h.split_ntask = h.mem.get<int>(std::max<size_t>(sbox.size(), 1));
    h.split_pbase = h.mem.get<int64_t>(std::max<size_t>(sbox.size(), 1));
    if (!sbox.empty()) {
        H3D_CUDA(cudaMemcpyAsync(h.split_box, sbox.data(), sbox.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        H3D_CUDA(cudaMemcpyAsync(h.split_task0, stask0.data(), sbox.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        H3D_CUDA(cudaMemcpyAsync(h.split_ntask, sntask.data(), sbox.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        H3D_CUDA(cudaMemcpyAsync(h.split_pbase, spbase.data(), sbox.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    }
    h.partial_elems = pel;
    h.partial = h.mem.alloc((size_t)std::max<int64_t>(pel, 4) * es);
    h.t = h.mem.alloc((size_t)std::max<int64_t>(h.sum_rank, 4) * es);
    h.xs = h.mem.alloc((size_t)std::max<int64_t>(h.N, 4) * es);
    h.nearbuf = h.mem.alloc((size_t)std::max<int64_t>(h.N, 4) * es);
    if (h.leaf_size <= kMaxLeafMR) {   // scratch of the multi-RHS product (kNQ columns per pass)
        h.xs_mr = h.mem.alloc((size_t)std::max<int64_t>(h.N, 4) * kNQ * es);
        h.nearbuf_mr = h.mem.alloc((size_t)std::max<int64_t>(h.N, 4) * kNQ * es);
        h.t_mr = h.mem.alloc((size_t)std::max<int64_t>(h.sum_rank, 4) * kNQ * es);
        h.partial_mr = h.mem.alloc((size_t)std::max<int64_t>(pel, 4) * kNQ * es);
    }
    // highest priority: the near-field CTAs are dispatched ahead of the gather's
    int prio_lo = 0, prio_hi = 0;
    H3D_CUDA(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    H3D_CUDA(cudaStreamCreateWithPriority(&h.side_stream, cudaStreamNonBlocking, prio_hi));
    H3D_CUDA(cudaEventCreateWithFlags(&h.ev_fork, cudaEventDisableTiming));
    H3D_CUDA(cudaEventCreateWithFlags(&h.ev_join, cudaEventDisableTiming));

    // transpose partials: per level l < L, per leaf z, R of its ancestor
    const int L = h.L, nleaf = h.nleaf;
    std::vector<int> anc((size_t)std::max(1, L) * nleaf);
    if (L > 0)
        H3D_CUDA(cudaMemcpyAsync(anc.data(), h.leaf_anc, anc.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
    H3D_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> tpb((size_t)std::max(1, L) * nleaf, 0);
    int64_t tel = 0;
    std::vector<int> tsb, tsl;
    for (int l = 1; l < L; ++l) {
        for (int z = 0; z < nleaf; ++z) {
            tpb[(size_t)(l - 1) * nleaf + z] = tel;
            tel += R[anc[(size_t)(l - 1) * nleaf + z]];
        }
        for (int64_t g = h.box_off[l]; g < h.box_off[l + 1]; ++g)
            if (R[g] > 0) { tsb.push_back((int)g); tsl.push_back(l); }
    }
    h.tp_base = h.mem.get<int64_t>(tpb.size());
    H3D_CUDA(cudaMemcpyAsync(h.tp_base, tpb.data(), tpb.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    h.tpartial_elems = tel;
    h.tpartial = h.mem.alloc((size_t)std::max<int64_t>(tel, 4) * es);
    h.nsplit_T = (int)tsb.size();
    h.tsplit_box = h.mem.get<int>(std::max<size_t>(tsb.size(), 1));
    h.tsplit_level = h.mem.get<int>(std::max<size_t>(tsb.size(), 1));
    if (!tsb.empty()) {
        H3D_CUDA(cudaMemcpyAsync(h.tsplit_box, tsb.data(), tsb.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        H3D_CUDA(cudaMemcpyAsync(h.tsplit_level, tsl.data(), tsl.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    H3D_CUDA(cudaStreamSynchronize(s));
}

int matvec_passes(const Handle &h, int nrhs, bool transpose) {
    if (use_wide(h, nrhs, transpose)) return (nrhs + kNQW - 1) / kNQW;
    if (nrhs > 1 && !transpose && h.leaf_size <= kMaxLeafMR) return (nrhs + kNQ - 1) / kNQ;
    return nrhs;
}

void run_matvec(Handle &h, const void *x, void *y, int nrhs, bool transpose, cudaStream_t s, cudaEvent_t *ev) {
    const int64_t n = h.N;
    if (use_wide(h, nrhs, transpose)) {
        ensure_wide_scratch(h, s);
        for (int q0 = 0, b = 0; q0 < nrhs; q0 += kNQW, ++b)
            matvec_wide(h, (const float *)x, (float *)y, q0, std::min(kNQW, nrhs - q0), s, ev ? ev + 5 * b : nullptr);
        return;
    }
    if (nrhs > 1 && !transpose && h.leaf_size <= kMaxLeafMR) {
        for (int q0 = 0, b = 0; q0 < nrhs; q0 += kNQ, ++b) {
            const int nq = std::min(kNQ, nrhs - q0);
            cudaEvent_t *e = ev ? ev + 5 * b : nullptr;
            if (h.prec == H3D_FP64) matvec_mr<double>(h, (const double *)x, (double *)y, q0, nq, s, e);
            else matvec_mr<float>(h, (const float *)x, (float *)y, q0, nq, s, e);
        }
        return;
    }
    for (int c = 0; c < nrhs; ++c) {
        cudaEvent_t *e = ev ? ev + 5 * c : nullptr;
        if (h.prec == H3D_FP64)
            matvec_one<double>(h, (const double *)x + (size_t)c * n, (double *)y + (size_t)c * n, transpose, s, e);
        else
            matvec_one<float>(h, (const float *)x + (size_t)c * n, (float *)y + (size_t)c * n, transpose, s, e);
    }
}

}  // namespace h3d
