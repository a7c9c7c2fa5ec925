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

#include <cuda.h>
#include <cudaTypedefs.h>

#include "h3d_async.cuh"
#include "h3d_ff.cuh"
#include "h3d_internal.cuh"
#include "h3d_stream.cuh"

namespace h3d {

namespace {

constexpr int64_t kTaskElems = 1 << 18;   // factor entries streamed by one gather task
// 32-column path: rows per gather task (the partial sums of split boxes cost
// 32 columns of traffic each, so its tasks are tall)
constexpr int kTaskRowsW = 4096;

template <class T>
__global__ void k_permute_in(const T *__restrict__ x, const int *__restrict__ perm, int64_t n, T *__restrict__ xs) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) xs[i] = x[perm[i]];
}

// A7 over the host-built task list: one task per CTA
template <class T>
__global__ void __launch_bounds__(kGatherThreads) k_gather(GatherArgs G, const T *__restrict__ V,
                                                           const T *__restrict__ xs, T *__restrict__ t,
                                                           T *__restrict__ partial) {
    __shared__ T xsm[kTaskMaxRows];
    __shared__ T red[kGatherThreads * Vec<T>::W];
    gather_task<T, kGatherThreads, 4, false>(G, blockIdx.x, V, xs, t, partial, xsm, red);
}

template <class T>
__global__ void k_reduce_partials(SplitArgs S, const T *__restrict__ partial, T *__restrict__ t) {
    reduce_split<T, false>(S, blockIdx.x, blockDim.x, partial, t);
}

// A8 + A9: one CTA per leaf
template <class T>
__global__ void __launch_bounds__(kLeafThreads) k_leaf(LeafArgs A, const T *__restrict__ U, const T *__restrict__ t,
                                                       const T *__restrict__ nearbuf, T *__restrict__ y) {
    extern __shared__ __align__(128) unsigned char stage[];   // kStages * kChunkBytes
    __shared__ __align__(8) uint64_t bars[kStages];
    __shared__ ChunkPlan P;
    __shared__ T red[kLeafThreads * Vec<T>::W];
    if (threadIdx.x == 0) {
        for (int q = 0; q < kStages; ++q) mbar_init(&bars[q], 1);
        mbar_fence_init();
    }
    uint32_t ring = 0;
    leaf_task<T, false>(A, blockIdx.x, U, t, nearbuf, y, stage, bars, P, red, ring);
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
        near_task<T>(A, z, xs, nearbuf, outsm, partsm, srcbuf);
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
// of up to kMaxLeafW points.  Right-hand sides, t and the near field are kept
// point-major (32 values per point / column); the factor products run on the
// tensor cores (k_tc_stream below), the near field on CUDA cores.
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

// sum of the row-task partials of split box blockIdx.y, columns
// [8 blockIdx.x, 8 blockIdx.x + 8): one thread per (column, right-hand side),
// so that every split box spreads over many CTAs
constexpr int kRedColsW = 8;
__global__ void __launch_bounds__(kRedColsW * kNQW) k_reduce_partials_w(SplitArgs S, const float *__restrict__ partial,
                                                                        float *__restrict__ t) {
    const int q = blockIdx.y;
    const int Y = S.box[q], R = S.Rv[Y];
    const int c = blockIdx.x * kRedColsW + (threadIdx.x >> 5), j = threadIdx.x & 31;
    if (c >= R) return;
    const int nt = S.ntask[q], ld = S.ldv[Y];
    const int64_t pb = S.pbase[q], vc0 = S.vcol0[Y];
    const float *p = partial + (pb + c) * kNQW + j;
    const int64_t step = (int64_t)ld * kNQW;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    int k = 0;
    for (; k + 4 <= nt; k += 4) {   // four loads in flight
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] += p[(k + u) * step];
    }
    for (; k < nt; ++k) v[0] += p[k * step];
    t[S.map_v[vc0 + c] * kNQW + j] = (v[0] + v[1]) + (v[2] + v[3]);
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
                // plain FMAs over the staged sources (at most CAP / S per thread),
                // then one compensated addition per right-hand side
                float bs[kNQW];
#pragma unroll
                for (int q = 0; q < kNQW; ++q) bs[q] = 0.f;
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
                        bs[4 * u] = fmaf(kij, b.x, bs[4 * u]);
                        bs[4 * u + 1] = fmaf(kij, b.y, bs[4 * u + 1]);
                        bs[4 * u + 2] = fmaf(kij, b.z, bs[4 * u + 2]);
                        bs[4 * u + 3] = fmaf(kij, b.w, bs[4 * u + 3]);
                    }
                }
#pragma unroll
                for (int q = 0; q < kNQW; ++q) acc[q].add(bs[q]);
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

// ===========================================================================
// Factor products of 32 right-hand sides on the tensor cores (tcgen05,
// kind::tf32, 3xTF32 split precision): one warp-specialised persistent kernel
// for both sides of the far field.
//   gather (kLeaf = false): T_Y(c, q) = sum_r V_Y(r, c) x(r, q), i.e.
//     D[M = 128 columns c of V][N] += A[M][K = rows r] B[K][N];
//     a work item is one gather task (source box, row range) x 128 columns.
//   leaf (kLeaf = true): y(i, q) = sum over levels, columns c of U_panel(i, c) t_A(c, q),
//     D[M = 128 rows][N] += A[M][K = c] B[K][N], plus the near field.  A work item
//     is a tile of sibling leaves (same parent) whose rows fit in 128: their
//     ancestors at levels 1..L-1 are shared, so each of those panels' K range is
//     one stage sequence for the whole tile (every leaf's rows stacked in M, one t
//     chunk in B); each leaf's own level-L panel then runs with the other leaves'
//     rows zero.
// Each item is cut into stages of up to kTsK = 32 K values (4 MMA K steps).
//  * warp 0, the producer, walks the items (descriptions of the next 32 gather
//    items are loaded while the current ones are issued) and fills a ring of
//    kTsSlots slots with TMA: the gather's V tile in one 2-D tensor copy from the
//    source box's tensor map, the leaf's U chunks in one bulk copy per leaf, and
//    the B tile (x or t rows, contiguous) in one bulk copy; full / empty mbarriers
//    per slot.
//  * warps 2-9, the converters, split each value into tf32 hi + lo (the tensor
//    core truncates FP32 operands, so both parts are rounded here): A straight
//    into tensor memory (lane = M row, one column per K value), B as one N = 64
//    operand [hi | lo] of K-major core matrices in shared memory (8 rows x 16
//    bytes; LBO 128 B along K, SBO 1024 B along N; K step j starts 256 B
//    further).  They drain the accumulators of the stage two behind into
//    registers.  Two warps share each quadrant of TMEM lanes: each converts half
//    of the stage's K values and drains half of the 32 right-hand sides.
//  * one thread of warp 1 issues a stage's MMAs, per K step
//      A_hi x [B_hi | B_lo]  (N = 64) -> the stage's main | first correction
//      A_lo x B_hi           (N = 32) -> the item's second correction,
//    then commits them to the stage's operand mbarrier.
// The tensor core's FP32 accumulation is biased (its error grows about one ulp per
// accumulated MMA), so each stage's main accumulator goes into a compensated FP32
// sum in registers as soon as the stage completes; the first correction is
// summed plainly per stage and the second stays in TMEM for the whole item (both
// are 2^-11 of the main term).
// Every wait is bounded.  A wait that gives up raises the CTA's abort flag, every
// role leaves its loop, copies and MMAs in flight are waited for (bounded), the
// error word is set and TMEM is freed.
constexpr int kTsConv = 256;                           // converter threads
constexpr int kTsThreads = 64 + kTsConv;
constexpr int kTsSlots = 8;
constexpr int kTsK = 32;                               // K values per stage
constexpr int kTsBOp = 32 * kTsK * 4;                  // B_hi or B_lo (32 x 32 tf32), 4 KB
constexpr int kTsBBuf = 2 * kTsBOp;                    // [B_hi | B_lo] as one N = 64 operand
constexpr int kTsSlotA = 128 * kTsK * 4;               // raw A tile
constexpr int kTsSlotB = 32 * kTsK * 4;                // raw B tile
constexpr int kTsSlot = kTsSlotA + kTsSlotB;
constexpr size_t kTsDynSmem = (size_t)kTsSlots * kTsSlot + 2 * (size_t)kTsBBuf + 128;
constexpr int kTcCols = 128;                           // gather: V columns per item
constexpr int kTileLeaves = 8;                         // leaves per far-field tile (siblings)
// tensor memory columns (512 allocated; one CTA per SM)
constexpr uint32_t kTmMain = 0;     // 2 stage sets x 64: main (32) | first correction (32)
constexpr uint32_t kTmCorr = 128;   // 2 item sets x 32: second correction
constexpr uint32_t kTmA = 256;      // 2 stage sets x 64: A_hi (32) | A_lo (32)

struct TsArgs {
    const TcGatherItem *gitems;
    const unsigned char *tmaps;   // CUtensorMap[], 128 bytes each
    const int2 *tiles;
    const float *V, *xs;
    float *t, *partial;
    const int64_t *map_v;
    LeafArgs A;
    const float *U, *tl, *nearbuf;
    float *y;
    int64_t n;
    int q0, nq;
    int nitems;               // gather items or leaf tiles
    int *err;
};

struct TsMeta {               // one per ring slot, written by the producer
    int nk;                   // K values of the stage; 0: an item without far field; -1: end
    int first, last;          // first / last stage of its item
    int sel;                  // leaf: -1 = every row of the tile is live, else the one live leaf
    int ncols, to_t;          // gather: valid columns, output to t (1) or partial (0)
    int z0, nl;               // leaf: first leaf of the tile, leaves
    int ld[kTileLeaves], off[kTileLeaves];   // leaf: rows and first tile row per leaf
    int64_t idx[kTcCols];     // gather, last stage: output row per column
};

struct TsOpMeta {             // per operand buffer, converters -> MMA issuer
    int nks, first, corr;     // K steps (-1: end), first stage of its item, correction set
};

// byte offset of element (row `n`, k) in a K-major operand of kTsK values
__device__ __forceinline__ int kmajor_off(int n, int k) {
    return ((n >> 3) << 10) + ((k >> 2) << 7) + ((n & 7) << 4) + ((k & 3) << 2);
}

template <bool kLeaf>
__global__ void __launch_bounds__(kTsThreads, 1) k_tc_stream(TsArgs P) {
    extern __shared__ unsigned char dsm_raw[];
    __shared__ __align__(8) uint64_t full[kTsSlots], empty[kTsSlots], opfull[2], opempty[2];
    __shared__ TsMeta meta[kTsSlots];
    __shared__ TsOpMeta opm[2];
    __shared__ int abort_flag;
    __shared__ uint32_t tmem_base;
    // producer-private plan of the current leaf tile
    __shared__ const float *pl_tl[kMaxDepth + 1], *pl_tL[kTileLeaves];
    __shared__ int64_t pl_ub[kMaxDepth + 1], pl_lplo[kMaxDepth + 1], pl_lp[kTileLeaves], pl_ubL[kTileLeaves];
    __shared__ int pl_R[kMaxDepth + 1], pl_RL[kTileLeaves], pl_ld[kTileLeaves], pl_off[kTileLeaves];
    unsigned char *ring = dsm_raw + ((128 - (smem_addr(dsm_raw) & 127)) & 127);
    unsigned char *bops = ring + (size_t)kTsSlots * kTsSlot;   // two [B_hi | B_lo] operands
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int *abort = &abort_flag;
    if (warp == 0) tmem_alloc(&tmem_base, 512);
    if (tid == 32) {
        for (int i = 0; i < kTsSlots; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kTsConv / 32);   // one arrival per converter warp
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&opfull[i], kTsConv / 32);
            mbar_init(&opempty[i], 1);
        }
        abort_flag = 0;
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        int s = 0;
        bool ok = true;
        auto acquire = [&](int slot) -> bool {   // wait until the converters released the slot
            if (s < kTsSlots) return true;
            return mbar_wait_or_abort(&empty[slot], (uint32_t)(((s / kTsSlots) - 1) & 1), abort);
        };
        if constexpr (!kLeaf) {
            // lane j holds the description of item base + j * gridDim.x; the next 32
            // are loaded while these are issued
            const int G = gridDim.x;
            TcGatherItem mine{}, nextb{};
            int base = blockIdx.x;
            if (base + lane * G < P.nitems) mine = P.gitems[base + lane * G];
            for (; base < P.nitems && ok; base += 32 * G) {
                if (base + 32 * G + lane * G < P.nitems) nextb = P.gitems[base + 32 * G + lane * G];
                for (int j = 0; j < 32 && ok; ++j) {
                    if (base + j * G >= P.nitems) break;
                    const int64_t gx = __shfl_sync(0xffffffffu, mine.x, j);
                    const int64_t go = __shfl_sync(0xffffffffu, mine.o, j);
                    const int tmap = __shfl_sync(0xffffffffu, mine.tmap, j);
                    const int c_lo = __shfl_sync(0xffffffffu, mine.c_lo, j);
                    const int r0 = __shfl_sync(0xffffffffu, mine.r0, j);
                    const int nrows = __shfl_sync(0xffffffffu, mine.nrows, j);
                    const int ncols = __shfl_sync(0xffffffffu, mine.ncols, j);
                    const int to_t = __shfl_sync(0xffffffffu, mine.to_t, j);
                    const unsigned char *tm = P.tmaps + 128 * (size_t)tmap;
                    const float *xsrc = P.xs + gx * kNQW;
                    for (int r = 0; r < nrows; r += kTsK) {
                        const int nk = min(kTsK, nrows - r), slot = s % kTsSlots;
                        if (!(ok = acquire(slot))) break;
                        TsMeta &M = meta[slot];
                        const bool last = r + kTsK >= nrows;
                        if (lane == 0) {
                            M.nk = nk;
                            M.first = r == 0;
                            M.last = last;
                            M.ncols = ncols;
                            M.to_t = to_t;
                        }
                        if (last) {   // output rows: copied asynchronously, tracked by the slot's barrier
#pragma unroll
                            for (int q = 0; q < kTcCols / 32; ++q) {
                                const int mc = lane + 32 * q;
                                if (mc >= ncols) M.idx[mc] = -1;
                                else if (to_t) cp_async8(&M.idx[mc], P.map_v + go + mc);
                                else M.idx[mc] = go + mc;
                            }
                            cp_async_arrive(&full[slot]);
                        }
                        __syncwarp();   // the lanes' stores are ordered before lane 0's release
                        if (lane == 0) {
                            unsigned char *sa = ring + (size_t)slot * kTsSlot;
                            // the tensor copy always moves the whole 32 x 128 box (zero outside the factor)
                            mbar_arrive_expect_tx(&full[slot], (uint32_t)(kTsSlotA + nk * kNQW * 4));
                            tma_load_2d(sa, tm, c_lo, r0 + r, &full[slot]);
                            bulk_copy_g2s(sa + kTsSlotA, xsrc + (int64_t)r * kNQW, (uint32_t)(nk * kNQW * 4),
                                          &full[slot]);
                        }
                        __syncwarp();
                        ++s;
                    }
                }
                mine = nextb;
            }
        } else {
            const LeafArgs &A = P.A;
            const int L = A.L;
            for (int it = blockIdx.x; it < P.nitems && ok; it += gridDim.x) {
                const int2 tile = P.tiles[it];
                const int z0 = tile.x, nl = tile.y;
                __syncwarp();   // every lane is done with the previous tile's plan
                const int ld = lane < nl ? A.leaf_ld[z0 + lane] : 0;
                int off = ld;   // inclusive prefix of the rows over the warp
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, off, d);
                    if (lane >= d) off += v;
                }
                if (lane < nl) {   // this tile's leaves: rows, tile offset, own (level-L) panel
                    const int z = z0 + lane;
                    pl_ld[lane] = ld;
                    pl_off[lane] = off - ld;
                    pl_lp[lane] = A.leaf_lp[z];
                    if (L > 0) {
                        const int Zg = A.leaf_anc[(int64_t)(L - 1) * A.nleaf + z];
                        pl_RL[lane] = A.R[Zg];
                        pl_ubL[lane] = A.ubase[Zg] + (A.leaf_lp[z] - A.leaf_lp[A.leaf_lo[Zg]]) * A.R[Zg];
                        pl_tL[lane] = P.tl + A.tbase[Zg] * kNQW;
                    } else {
                        pl_RL[lane] = 0;
                    }
                }
                if (lane >= 1 && lane < L) {   // shared ancestors at levels 1 .. L-1
                    const int Ag = A.leaf_anc[(int64_t)(lane - 1) * A.nleaf + z0];
                    pl_R[lane] = A.R[Ag];
                    pl_ub[lane] = A.ubase[Ag];
                    pl_lplo[lane] = A.leaf_lp[A.leaf_lo[Ag]];
                    pl_tl[lane] = P.tl + A.tbase[Ag] * kNQW;
                }
                __syncwarp();
                int nst = 0;
                for (int l = 1; l < L; ++l) nst += (pl_R[l] + kTsK - 1) / kTsK;
                for (int g = 0; g < nl; ++g) nst += (pl_RL[g] + kTsK - 1) / kTsK;
                auto stage = [&](int st, int nk, int sel) -> bool {
                    const int slot = s % kTsSlots;
                    if (!acquire(slot)) return false;
                    if (lane == 0) {
                        TsMeta &M = meta[slot];
                        M.nk = nk;
                        M.first = st == 0;
                        M.last = st == max(nst, 1) - 1;
                        M.sel = sel;
                        M.z0 = z0;
                        M.nl = nl;
                        for (int g = 0; g < kTileLeaves; ++g) {
                            M.ld[g] = g < nl ? pl_ld[g] : 0;
                            M.off[g] = g < nl ? pl_off[g] : 128;
                        }
                    }
                    __syncwarp();
                    if (lane == 0) {   // its arrive releases the meta it wrote
                        uint32_t bytes = (uint32_t)(nk * kNQW * 4);
                        for (int g = 0; g < nl; ++g)
                            if (sel < 0 || sel == g) bytes += (uint32_t)(nk * pl_ld[g] * 4);
                        if (nk > 0) mbar_arrive_expect_tx(&full[slot], bytes);
                        else mbar_arrive(&full[slot]);
                    }
                    __syncwarp();
                    ++s;
                    return true;
                };
                int st = 0;
                for (int l = 1; l < L && ok; ++l) {
                    const int R = pl_R[l];
                    for (int c0 = 0; c0 < R; c0 += kTsK, ++st) {
                        const int nk = min(kTsK, R - c0);
                        unsigned char *sa = ring + (size_t)(s % kTsSlots) * kTsSlot;
                        uint64_t *bar = &full[s % kTsSlots];
                        if (!(ok = stage(st, nk, -1))) break;
                        if (lane < nl)
                            bulk_copy_g2s(sa + 128 * pl_off[lane],
                                          P.U + pl_ub[l] + (pl_lp[lane] - pl_lplo[l]) * R + (int64_t)c0 * pl_ld[lane],
                                          (uint32_t)(nk * pl_ld[lane] * 4), bar);
                        if (lane == 31)
                            bulk_copy_g2s(sa + kTsSlotA, pl_tl[l] + (int64_t)c0 * kNQW, (uint32_t)(nk * kNQW * 4), bar);
                    }
                }
                for (int g = 0; g < nl && ok; ++g) {
                    const int R = pl_RL[g];
                    for (int c0 = 0; c0 < R; c0 += kTsK, ++st) {
                        const int nk = min(kTsK, R - c0);
                        unsigned char *sa = ring + (size_t)(s % kTsSlots) * kTsSlot;
                        uint64_t *bar = &full[s % kTsSlots];
                        if (!(ok = stage(st, nk, g))) break;
                        if (lane == 0)
                            bulk_copy_g2s(sa + 128 * pl_off[g], P.U + pl_ubL[g] + (int64_t)c0 * pl_ld[g],
                                          (uint32_t)(nk * pl_ld[g] * 4), bar);
                        if (lane == 31)
                            bulk_copy_g2s(sa + kTsSlotA, pl_tL[g] + (int64_t)c0 * kNQW, (uint32_t)(nk * kNQW * 4), bar);
                    }
                }
                if (ok && nst == 0) ok = stage(0, 0, -1);   // no far field: the tile still reaches its output
            }
        }
        if (ok) {   // end marker
            const int slot = s % kTsSlots;
            if ((ok = acquire(slot))) {
                if (lane == 0) {
                    meta[slot].nk = -1;
                    meta[slot].first = meta[slot].last = 0;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[slot]);
            }
        }
        if (!ok && lane == 0)   // copies still in flight land before the CTA leaves
            for (int j = max(0, s - kTsSlots); j < s; ++j) mbar_wait(&full[j % kTsSlots], (uint32_t)((j / kTsSlots) & 1));
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t id64 = umma_idesc_tf32(128, 2 * kNQW), id32 = umma_idesc_tf32(128, kNQW);
            int s = 0;
            for (;; ++s) {
                const int b = s & 1;
                if (!mbar_wait_or_abort(&opfull[b], (uint32_t)((s >> 1) & 1), abort)) break;
                tc_fence_after();
                const TsOpMeta om = opm[b];
                if (om.nks < 0) break;
                const uint32_t bbase = smem_addr(bops + b * kTsBBuf);
                const uint32_t dmain = tmem + kTmMain + 64u * (uint32_t)b;
                const uint32_t dcorr = tmem + kTmCorr + 32u * (uint32_t)om.corr;
                const uint32_t ahi = tmem + kTmA + 64u * (uint32_t)b, alo = ahi + 32u;
                for (int j = 0; j < om.nks; ++j) {
                    const uint64_t bd = umma_desc(bbase + 256u * (uint32_t)j, 128, 1024);
                    umma_tf32_ts(dmain, ahi + 8u * (uint32_t)j, bd, id64, j > 0 ? 1u : 0u);
                    umma_tf32_ts(dcorr, alo + 8u * (uint32_t)j, bd, id32, (j > 0 || !om.first) ? 1u : 0u);
                }
                umma_commit(&opempty[b]);
            }
            if (*abort)   // this thread's MMAs finish before TMEM is freed
                for (int j = max(0, s - 2); j < s; ++j) mbar_wait(&opempty[j & 1], (uint32_t)((j >> 1) & 1));
        }
    } else {
        // ------------------------------------------------------------ converters
        const int c = warp - 2;                                  // 0..7
        const int m = ((warp & 3) << 5) | lane;                  // M row = TMEM lane
        const int hk = (c >> 2) * (kTsK / 2);                    // this warp's half of the K values
        const int hq = (c >> 2) * (kNQW / 2);                    // and of the right-hand sides
        const uint32_t tlane = (uint32_t)((warp & 3) << 5) << 16;
        const int kb = 4 * c;                                    // B: K values kb..kb+3 of right-hand side lane
        constexpr int QH = kNQW / 2;
        Acc<float> acc[QH];
        float cacc[QH];
#pragma unroll
        for (int q = 0; q < QH; ++q) cacc[q] = 0.f;
        struct Pend {   // a stage waiting for its drain
            int nk, last, mma, corr;   // K values, last of its item, item had MMAs, correction set
            int a, i;                  // gather: output to t; leaf: this row's leaf (-1: none), row in leaf
            int64_t o;                 // gather: output row of this thread's column (-1: none)
        };
        Pend p1{0, 0, 0, 0, 0, 0, -1}, p2 = p1;
        int item = 0, item_mma = 0;    // items started, current item had MMAs
        int lg = -1, li = 0, lbase = 0, lstride = 0;   // leaf: this row's leaf, row, slot base, stride
        // a completed stage: its main accumulator into the compensated sums, its
        // first correction into the plain ones; the item's output after its last stage
        auto drain = [&](const Pend &pd, int set) {
            if (pd.nk > 0) {
                float v[QH], w[QH];
                const uint32_t dm = tmem + tlane + kTmMain + 64u * (uint32_t)set + (uint32_t)hq;
                tmem_ld16x2(dm, dm + 32u, v, w);
#pragma unroll
                for (int q = 0; q < QH; ++q) {
                    acc[q].add(v[q]);
                    cacc[q] += w[q];
                }
            }
            if (!pd.last) return;
            float cr[QH];
            if (pd.mma) {
                tmem_ld16(tmem + tlane + kTmCorr + 32u * (uint32_t)pd.corr + (uint32_t)hq, cr);
            } else {
#pragma unroll
                for (int q = 0; q < QH; ++q) cr[q] = 0.f;
            }
#pragma unroll
            for (int q = 0; q < QH; ++q) cr[q] += cacc[q];
            if constexpr (!kLeaf) {
                if (pd.o >= 0) {
                    float *o = (pd.a ? P.t : P.partial) + pd.o * kNQW + hq;
#pragma unroll
                    for (int q = 0; q < QH; q += 4)
                        *reinterpret_cast<float4 *>(o + q) =
                            make_float4(acc[q].get() + cr[q], acc[q + 1].get() + cr[q + 1], acc[q + 2].get() + cr[q + 2],
                                        acc[q + 3].get() + cr[q + 3]);
                }
            } else if (pd.a >= 0) {
                const int Zg = (int)(P.A.offL + pd.a);
                const int zs = P.A.box_start[Zg];
                if (pd.i < P.A.box_end[Zg] - zs) {
                    const int64_t o = P.A.perm[zs + pd.i];
                    const float *nb = P.nearbuf + (int64_t)(zs + pd.i) * kNQW + hq;
#pragma unroll
                    for (int q = 0; q < QH; ++q)
                        if (hq + q < P.nq) P.y[(int64_t)(P.q0 + hq + q) * P.n + o] = (acc[q].get() + cr[q]) + nb[q];
                }
            }
#pragma unroll
            for (int q = 0; q < QH; ++q) {
                acc[q] = Acc<float>{};
                cacc[q] = 0.f;
            }
        };

        for (int s = 0;; ++s) {
            const int slot = s % kTsSlots, b = s & 1;
            if (!mbar_wait_or_abort(&full[slot], (uint32_t)((s / kTsSlots) & 1), abort)) break;
            const TsMeta &M = meta[slot];
            const int nk = M.nk;
            if (s >= 2) {   // the MMAs of stage s-2 are done: its operands and accumulator are free
                if (!mbar_wait_or_abort(&opempty[b], (uint32_t)(((s - 2) >> 1) & 1), abort)) break;
                tc_fence_after();
                drain(p2, b);
            }
            if (nk < 0) {   // end: stop the issuer, drain the last stage
                if (c == 0 && lane == 0) opm[b].nks = -1;
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&opfull[b]);
                if (s >= 1) {
                    if (!mbar_wait_or_abort(&opempty[b ^ 1], (uint32_t)(((s - 1) >> 1) & 1), abort)) break;
                    tc_fence_after();
                    drain(p1, b ^ 1);
                }
                break;
            }
            if (M.first) {
                ++item;
                item_mma = 0;
                if constexpr (kLeaf) {   // this row's leaf in the new tile
                    lg = -1;
                    for (int g = 0; g < M.nl; ++g)
                        if (m >= M.off[g] && m < M.off[g] + M.ld[g]) lg = g;
                    if (lg >= 0) {
                        li = m - M.off[lg];
                        lbase = 32 * M.off[lg] + li;
                        lstride = M.ld[lg];
                    }
                }
            }
            if (nk > 0) item_mma = 1;
            const int corr = item & 1;
            Pend cur{nk, M.last, item_mma, corr, 0, 0, -1};
            if (nk > 0) {
                const float *ta = reinterpret_cast<const float *>(ring + (size_t)slot * kTsSlot);
                const float *tb = ta + kTsSlotA / 4;
                bool live;
                int base, stride;
                if constexpr (!kLeaf) {   // A(m, k) = V tile row k, column m (rows of 128 floats)
                    live = m < M.ncols;
                    base = m;
                    stride = kTcCols;
                } else {                  // A(m, k) = the leaf's U chunk column k, row li
                    live = lg >= 0 && (M.sel < 0 || M.sel == lg);
                    base = lbase;
                    stride = lstride;
                }
                float h[16], l[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int k = hk + u;
                    split_tf32((live && k < nk) ? ta[base + k * stride] : 0.f, h[u], l[u]);
                }
                const uint32_t acol = tmem + tlane + kTmA + 64u * (uint32_t)b + (uint32_t)hk;
                tmem_st16(acol, h);
                tmem_st16(acol + 32u, l);
                {
                    float bh[4], bl[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = kb + u;
                        split_tf32(k < nk ? tb[k * kNQW + lane] : 0.f, bh[u], bl[u]);
                    }
                    unsigned char *bbuf = bops + b * kTsBBuf;
                    const int off = kmajor_off(lane, kb);
                    *reinterpret_cast<float4 *>(bbuf + off) = make_float4(bh[0], bh[1], bh[2], bh[3]);
                    *reinterpret_cast<float4 *>(bbuf + kTsBOp + off) = make_float4(bl[0], bl[1], bl[2], bl[3]);
                }
                tmem_st_wait();
            }
            if (M.last) {
                if constexpr (!kLeaf) {
                    cur.a = M.to_t;
                    cur.o = M.idx[m];
                } else {
                    cur.a = lg >= 0 ? M.z0 + lg : -1;
                    cur.i = li;
                }
            }
            if (c == 0 && lane == 0) opm[b] = TsOpMeta{(nk + 7) >> 3, M.first, corr};
            // every lane: its B stores visible to the tensor core, its TMEM stores
            // ordered before the barrier; then one arrival per warp on each barrier
            fence_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&empty[slot]);   // the warp is done with the slot
                mbar_arrive(&opfull[b]);
            }
            p2 = p1;
            p1 = cur;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (*abort && tid == 0) *P.err = H3D_ERR_TIMEOUT;
    if (warp == 0) tmem_dealloc(tmem, 512);
}

unsigned gridn(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

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
        const bool sym = h.symmetric();
        if (sym) sym_product(h, xs, 1, s, ev ? ev[2] : nullptr);   // the fused pairs, beside the gather
        if (h.ngtask > 0) {
            GatherArgs G{h.gtask, h.gtask_pbase, h.box_start, h.Rv, h.ldv, h.vbase, h.vcol0, h.map_v};
            k_gather<T><<<h.ngtask, kGatherThreads, 0, s>>>(G, (const T *)h.V, xs, t, (T *)h.partial);
        }
        if (ev && !sym) H3D_CUDA(cudaEventRecord(ev[2], s));
        if (h.nsplit > 0) {
            SplitArgs S{h.split_box, h.split_ntask, h.split_pbase, h.Rv, h.ldv, h.vcol0, h.map_v};
            k_reduce_partials<T><<<h.nsplit, 256, 0, s>>>(S, (const T *)h.partial, t);
        }
        H3D_CUDA(cudaStreamWaitEvent(s, h.ev_join, 0));
        if (sym) sym_finish(h, nearbuf, 1, s);
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
    TsArgs T{};
    T.gitems = h.tc_items;
    T.tmaps = (const unsigned char *)h.tc_tmaps;
    T.tiles = h.tc_tiles;
    T.V = (const float *)h.V;
    T.xs = xs;
    T.t = t;
    T.partial = (float *)h.partial_w;
    T.map_v = h.map_v;
    T.A = A;
    T.U = (const float *)h.U;
    T.tl = t;
    T.nearbuf = nearbuf;
    T.y = y;
    T.n = n;
    T.q0 = q0;
    T.nq = nq;
    T.err = h.d_async_err;
    if (h.ntc_items > 0) {
        T.nitems = h.ntc_items;
        k_tc_stream<false><<<std::min(h.ntc_items, num_sms()), kTsThreads, kTsDynSmem, s>>>(T);
    }
    if (ev) H3D_CUDA(cudaEventRecord(ev[2], s));
    if (h.nsplit_w > 0) {
        SplitArgs S{h.split_box_w, h.split_ntask_w, h.split_pbase_w, h.Rv, h.ldv, h.vcol0, h.map_v};
        const dim3 grid((unsigned)((h.max_rv_split_w + kRedColsW - 1) / kRedColsW), (unsigned)h.nsplit_w);
        k_reduce_partials_w<<<grid, kRedColsW * kNQW, 0, s>>>(S, (const float *)h.partial_w, t);
    }
    H3D_CUDA(cudaStreamWaitEvent(s, h.ev_join, 0));
    if (ev) H3D_CUDA(cudaEventRecord(ev[3], s));
    T.nitems = h.ntc_tiles;
    k_tc_stream<true><<<std::min(h.ntc_tiles, num_sms()), kTsThreads, kTsDynSmem, s>>>(T);
    if (ev) H3D_CUDA(cudaEventRecord(ev[4], s));
    H3D_LAUNCH_CHECK();
}

// scratch of the 32-column path, allocated by the first product that needs it
void ensure_wide_scratch(Handle &h, cudaStream_t s) {
    if (h.xs_w) return;
    H3D_CUDA(cudaStreamSynchronize(s));
    const size_t es = sizeof(float);
    void *xs = nullptr;   // xs_w last: it marks the scratch as made
    alloc_all(h.mem, {{&h.nearbuf_w, (size_t)std::max<int64_t>(h.N, 4) * kNQW * es},
                      {&h.t_w, (size_t)std::max<int64_t>(h.sum_rank, 4) * kNQW * es},
                      {&h.partial_w, (size_t)std::max<int64_t>(h.partial_elems_w, 4) * kNQW * es},
                      {&xs, (size_t)std::max<int64_t>(h.N, 4) * kNQW * es}});
    h.xs_w = xs;
}

bool use_wide(const Handle &h, int nrhs, bool transpose) {
    return nrhs > kNQ && !transpose && h.prec == H3D_FP32 && h.tf32 && h.leaf_size <= kMaxLeafW &&
           h.storage == H3D_STORE_FACTORS;
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
    const bool sym = h.symmetric();
    if (sym) sym_product(h, xs, kNQ, s, ev ? ev[2] : nullptr);   // the fused pairs, 8 columns, beside the gather
    if (h.ngtask > 0) {
        GatherArgs G{h.gtask, h.gtask_pbase, h.box_start, h.Rv, h.ldv, h.vbase, h.vcol0, h.map_v};
        k_gather_mr<T><<<h.ngtask, kGatherThreads, 0, s>>>(G, (const T *)h.V, xs, t, (T *)h.partial_mr);
    }
    if (ev && !sym) H3D_CUDA(cudaEventRecord(ev[2], s));
    if (h.nsplit > 0) {
        SplitArgs S{h.split_box, h.split_ntask, h.split_pbase, h.Rv, h.ldv, h.vcol0, h.map_v};
        k_reduce_partials_mr<T><<<h.nsplit, 256, 0, s>>>(S, (const T *)h.partial_mr, t);
    }
    H3D_CUDA(cudaStreamWaitEvent(s, h.ev_join, 0));
    if (sym) sym_finish(h, nearbuf, kNQ, s);
    if (ev) H3D_CUDA(cudaEventRecord(ev[3], s));
    k_leaf_mr<T><<<h.nleaf, kLeafThreads, kLeafDynSmem, s>>>(A, (const T *)h.U, t, nearbuf, y, n, q0, nq);
    if (ev) H3D_CUDA(cudaEventRecord(ev[4], s));
    H3D_LAUNCH_CHECK();
}

// ===========================================================================
// Skeleton storage (the paper's own, Sec. 4.1): per admissible block only the
// pivots and an LU factorisation of M = K(sigma,tau); a product recomputes
// K(sigma,Y) x_Y, solves with M and applies K(X,tau).  Entries are FP64: the
// solve's output carries the condition of M (up to ~1e7), which FP32 entries of
// K(X,tau) would turn into O(1) errors.

// 1/sqrt(d2) to FP64 accuracy without the FP64 square root or division
__device__ __forceinline__ double skel_rsqrt(double d2) {
    // FP32 seed y0 (|relative error| < 2^-21), then one third-order step of
    // y = y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3 e^2/8 + ...), e = 1 - d2 y0^2 (y0^2
    // exact in FP64); the neglected terms are below 2^-60
    const double y0 = (double)rsqrtf((float)d2);
    const double e = fma(-d2, y0 * y0, 1.0);
    return fma(y0 * e, fma(0.375, e, 0.5), y0);
}

// K(p_i, p_j) from the coordinate differences p_i - p_j
__device__ __forceinline__ double skel_kd(int kind, double kappa, double dx, double dy, double dz) {
    const double d2 = dx * dx + dy * dy + dz * dz;
    if (d2 == 0.0) return 0.0;
    const double ir = skel_rsqrt(d2);
    switch (kind) {
    case H3D_LAPLACE: return H3D_INV4PI * ir;
    case H3D_YUKAWA: return H3D_INV4PI * exp(-kappa * d2 * ir) * ir;
    case H3D_INV_R4: return (ir * ir) * (ir * ir);
    default: return cos(d2 * ir) * ir;
    }
}

__device__ __forceinline__ double skel_k(int kind, double kappa, const double *px, const double *py,
                                         const double *pz, int i, int j) {
    const double dx = px[i] - px[j], dy = py[i] - py[j], dz = pz[i] - pz[j];
    const double d2 = dx * dx + dy * dy + dz * dz;
    if (d2 == 0.0) return 0.0;
    const double ir = skel_rsqrt(d2);
    switch (kind) {
    case H3D_LAPLACE: return H3D_INV4PI * ir;
    case H3D_YUKAWA: return H3D_INV4PI * exp(-kappa * d2 * ir) * ir;
    case H3D_INV_R4: return (ir * ir) * (ir * ir);
    default: return cos(d2 * ir) * ir;
    }
}

struct SkelArgs {
    int kind;
    double kappa;
    const double *px, *py, *pz;
    const float4 *fh, *fl;    // float-float coordinates (FP32 handles, Laplace and 1/r^4)
    int64_t nblk;
    const int *blk_tgt, *blk_src, *box_start, *box_end, *rank, *sigma, *tau;
    const int64_t *piv_off, *lu_off;
    double *lu;
    int *lu_piv;
    double *sbuf, *cbuf;
    int mr;                   // largest rank (per-warp scratch stride)
    int cst;                  // columns per pass (cbuf stride per pivot)
    int *next;                // source-side pass: next block (zero before the launch)
    int ff;                   // LU factors, pivot sums and coefficients held as float-float pairs
    // large blocks: their pivot sums come from k_skel_rows (one warp per pivot)
    const int64_t *bigpo;     // per block: first slot in sbig, or -1
    double *sbig;             // kSkNQ values per pivot of the large blocks
};

// next block for a warp of a source-side pass: blocks in list order (largest,
// level 1, first) from one queue, so that a few large blocks do not leave the
// warps that drew them running long after the rest
__device__ __forceinline__ int64_t skel_next_block(const SkelArgs &S, int lane) {
    int b = 0;
    if (lane == 0) b = atomicAdd(S.next, 1);
    return __shfl_sync(0xffffffffu, b, 0);
}

constexpr int kSkThreads = 128;
constexpr int64_t kSkBig = 1 << 14;   // entries r x max(m, n) from which a block's pivot sums are spread over warps
constexpr int kSkLeafStage = 128;   // pivots staged per warp at a time (single-column leaf pass)

// M = K(sigma,tau) of every block, factored P M = L U in place (partial pivoting)
__global__ void __launch_bounds__(kSkThreads) k_skel_factor(SkelArgs S) {
    __shared__ int piv[kMaxRank];
    __shared__ int pmax;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int64_t b = blockIdx.x; b < S.nblk; b += gridDim.x) {
        const int r = S.rank[b];
        if (r == 0) continue;
        const int x0 = S.box_start[S.blk_tgt[b]], y0 = S.box_start[S.blk_src[b]];
        const int *sg = S.sigma + S.piv_off[b], *ta = S.tau + S.piv_off[b];
        double *M = S.lu + S.lu_off[b];
        for (int e = tid; e < r * r; e += kSkThreads) {
            const int k = e / r, l = e - k * r;
            M[e] = skel_k(S.kind, S.kappa, S.px, S.py, S.pz, x0 + sg[k], y0 + ta[l]);
        }
        for (int k = tid; k < r; k += kSkThreads) piv[k] = k;
        __syncthreads();
        for (int k = 0; k < r; ++k) {
            if (warp == 0) {
                double best = -1.0;
                int bi = k;
                for (int i = k + lane; i < r; i += 32) {
                    const double v = fabs(M[(size_t)i * r + k]);
                    if (v > best || (v == best && i < bi)) { best = v; bi = i; }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
                }
                if (lane == 0) pmax = bi;
            }
            __syncthreads();
            const int p = pmax;
            if (p != k) {
                for (int j = tid; j < r; j += kSkThreads) {
                    const double t = M[(size_t)k * r + j];
                    M[(size_t)k * r + j] = M[(size_t)p * r + j];
                    M[(size_t)p * r + j] = t;
                }
                if (tid == 0) {
                    const int ti = piv[k];
                    piv[k] = piv[p];
                    piv[p] = ti;
                }
            }
            __syncthreads();
            const double d = M[(size_t)k * r + k];
            for (int i = k + 1 + tid; i < r; i += kSkThreads) M[(size_t)i * r + k] /= d;
            __syncthreads();
            const int rem = r - k - 1;
            for (int e = tid; e < rem * rem; e += kSkThreads) {
                const int i = k + 1 + e / rem, j = k + 1 + e % rem;
                M[(size_t)i * r + j] -= M[(size_t)i * r + k] * M[(size_t)k * r + j];
            }
            __syncthreads();
        }
        if (S.ff)   // float-float factors for the float-float solves, the diagonal as its reciprocal
            for (int e = tid; e < r * r; e += kSkThreads) {
                const double v = (e % (r + 1) == 0) ? 1.0 / M[e] : M[e];
                const FF f = ff_from_double(v);
                *reinterpret_cast<float2 *>(M + e) = make_float2(f.h, f.l);
            }
        for (int k = tid; k < r; k += kSkThreads) S.lu_piv[S.piv_off[b] + k] = piv[k];
        __syncthreads();
    }
}

// up to kSkNQ right-hand sides per pass: each entry is evaluated once for all
constexpr int kSkNQ = 16;

// xs[i * nq + q] = x[(q0 + q) n + perm[i]]: the pass's columns, point-major
template <class T>
__global__ void k_skel_permute(const T *__restrict__ x, int64_t n, int q0, int nq, const int *__restrict__ perm,
                               T *__restrict__ xs) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * nq) return;
    const int64_t i = e / nq;
    const int q = (int)(e - i * nq);
    xs[e] = x[(int64_t)(q0 + q) * n + perm[i]];
}

// per block (one warp): s = K(sigma,Y) X_Y for the pass's nq <= NQ columns (each
// entry evaluated once), then C = U^{-1} L^{-1} P s with lane q solving column q.
// cbuf: kSkNQ values per pivot; sbuf: a scratch of max_rank x kSkNQ per warp.
// float-float values stored in the 8 bytes of a double slot
__device__ __forceinline__ FF ld_ff(const double *p) {
    const float2 v = *reinterpret_cast<const float2 *>(p);
    return FF{v.x, v.y};
}
__device__ __forceinline__ void st_ff(double *p, FF v) { *reinterpret_cast<float2 *>(p) = make_float2(v.h, v.l); }
// a - b c, renormalised (TwoSum of the result's two parts): the triangular
// solves cancel at nearly every step, and a low part left larger than the high
// part's last bit would then carry only single precision into the next step
__device__ __forceinline__ FF ff_fms(FF a, FF b, FF c) {
    const FF p = ff_mul(b, c);
    const FF t = ff_two_sum(a.h, -p.h);
    return ff_two_sum(t.h, __fadd_rn(__fsub_rn(a.l, p.l), t.l));
}
__device__ __forceinline__ FF ff_shfl(FF v, int src) {
    return FF{__shfl_sync(0xffffffffu, v.h, src), __shfl_sync(0xffffffffu, v.l, src)};
}

// Float-float solves with the float-float LU of one block (row-major r x r, L
// unit lower, the diagonal of U stored as its reciprocal; P M = L U, pv the row
// order).  s: pivot sums at stride kSkNQ; c: the result at stride cst.  With
// every intermediate renormalised, the solve's rounding acts like a relative
// perturbation of ~1e-14 of the factors, which changes the block's product by
// far less than the ACA tolerance, so the FP64 pipe is not needed here.
//   c = U^{-1} L^{-1} P s           (forward product)
template <int NQ>
__device__ __forceinline__ void ff_solve(const double *M, const int *pv, int r, const double *sv, double *cv, int cst,
                                         int nq, int lane) {
    if (NQ == 1 && r <= 64) {   // lane k holds rows k and k + 32
        const int k0 = lane, k1 = lane + 32;
        FF z0 = k0 < r ? ld_ff(sv + (int64_t)pv[k0] * kSkNQ) : FF{0.f, 0.f};
        FF z1 = k1 < r ? ld_ff(sv + (int64_t)pv[k1] * kSkNQ) : FF{0.f, 0.f};
        for (int l = 0; l < r; ++l) {   // L z = P s
            const FF zl = ff_shfl(l < 32 ? z0 : z1, l & 31);
            if (k0 > l && k0 < r) z0 = ff_fms(z0, ld_ff(M + (size_t)k0 * r + l), zl);
            if (k1 > l && k1 < r) z1 = ff_fms(z1, ld_ff(M + (size_t)k1 * r + l), zl);
        }
        for (int l = r - 1; l >= 0; --l) {   // U c = z
            if (lane == (l & 31)) {
                if (l < 32) z0 = ff_mul(z0, ld_ff(M + (size_t)l * r + l));
                else z1 = ff_mul(z1, ld_ff(M + (size_t)l * r + l));
            }
            const FF cl = ff_shfl(l < 32 ? z0 : z1, l & 31);
            if (k0 < l) z0 = ff_fms(z0, ld_ff(M + (size_t)k0 * r + l), cl);
            if (k1 < l) z1 = ff_fms(z1, ld_ff(M + (size_t)k1 * r + l), cl);
        }
        if (k0 < r) st_ff(cv + (int64_t)k0 * cst, z0);
        if (k1 < r) st_ff(cv + (int64_t)k1 * cst, z1);
    } else if (NQ == 1) {   // the warp shares each dot product
        for (int k = 0; k < r; ++k) {
            FF acc{0.f, 0.f};
            for (int l = lane; l < k; l += 32) acc = ff_fma_acc(acc, ld_ff(M + (size_t)k * r + l), ld_ff(cv + (int64_t)l * cst));
            acc = ff_warp_sum(acc);
            if (lane == 0) st_ff(cv + (int64_t)k * cst, ff_fms(ld_ff(sv + (int64_t)pv[k] * kSkNQ), acc, FF{1.f, 0.f}));
            __syncwarp();
        }
        for (int k = r - 1; k >= 0; --k) {
            FF acc{0.f, 0.f};
            for (int l = k + 1 + lane; l < r; l += 32)
                acc = ff_fma_acc(acc, ld_ff(M + (size_t)k * r + l), ld_ff(cv + (int64_t)l * cst));
            acc = ff_warp_sum(acc);
            if (lane == 0)
                st_ff(cv + (int64_t)k * cst,
                      ff_mul(ff_fms(ld_ff(cv + (int64_t)k * cst), acc, FF{1.f, 0.f}), ld_ff(M + (size_t)k * r + k)));
            __syncwarp();
        }
    } else if (lane < nq) {   // lane q solves column q
        const int q = lane;
        for (int k = 0; k < r; ++k) {
            FF z = ld_ff(sv + (int64_t)pv[k] * kSkNQ + q);
            for (int l = 0; l < k; ++l) z = ff_fms(z, ld_ff(M + (size_t)k * r + l), ld_ff(cv + (int64_t)l * cst + q));
            st_ff(cv + (int64_t)k * cst + q, z);
        }
        for (int k = r - 1; k >= 0; --k) {
            FF z = ld_ff(cv + (int64_t)k * cst + q);
            for (int l = k + 1; l < r; ++l) z = ff_fms(z, ld_ff(M + (size_t)k * r + l), ld_ff(cv + (int64_t)l * cst + q));
            st_ff(cv + (int64_t)k * cst + q, ff_mul(z, ld_ff(M + (size_t)k * r + k)));
        }
    }
}

//   a = P^T L^{-T} U^{-T} u          (transpose product); sv is overwritten
template <int NQ>
__device__ __forceinline__ void ff_solve_T(const double *M, const int *pv, int r, double *sv, double *cv, int cst,
                                           int nq, int lane) {
    if (NQ == 1 && r <= 64) {
        const int k0 = lane, k1 = lane + 32;
        FF z0 = k0 < r ? ld_ff(sv + (int64_t)k0 * kSkNQ) : FF{0.f, 0.f};
        FF z1 = k1 < r ? ld_ff(sv + (int64_t)k1 * kSkNQ) : FF{0.f, 0.f};
        for (int l = 0; l < r; ++l) {   // U^T z = u
            if (lane == (l & 31)) {
                if (l < 32) z0 = ff_mul(z0, ld_ff(M + (size_t)l * r + l));
                else z1 = ff_mul(z1, ld_ff(M + (size_t)l * r + l));
            }
            const FF zl = ff_shfl(l < 32 ? z0 : z1, l & 31);
            if (k0 > l && k0 < r) z0 = ff_fms(z0, ld_ff(M + (size_t)l * r + k0), zl);
            if (k1 > l && k1 < r) z1 = ff_fms(z1, ld_ff(M + (size_t)l * r + k1), zl);
        }
        for (int l = r - 1; l >= 0; --l) {   // L^T w = z
            const FF wl = ff_shfl(l < 32 ? z0 : z1, l & 31);
            if (k0 < l) z0 = ff_fms(z0, ld_ff(M + (size_t)l * r + k0), wl);
            if (k1 < l) z1 = ff_fms(z1, ld_ff(M + (size_t)l * r + k1), wl);
        }
        if (k0 < r) st_ff(cv + (int64_t)pv[k0] * cst, z0);
        if (k1 < r) st_ff(cv + (int64_t)pv[k1] * cst, z1);
    } else if (NQ == 1) {
        for (int k = 0; k < r; ++k) {   // U^T z = u
            FF acc{0.f, 0.f};
            for (int l = lane; l < k; l += 32) acc = ff_fma_acc(acc, ld_ff(M + (size_t)l * r + k), ld_ff(sv + (int64_t)l * kSkNQ));
            acc = ff_warp_sum(acc);
            if (lane == 0)
                st_ff(sv + (int64_t)k * kSkNQ,
                      ff_mul(ff_fms(ld_ff(sv + (int64_t)k * kSkNQ), acc, FF{1.f, 0.f}), ld_ff(M + (size_t)k * r + k)));
            __syncwarp();
        }
        for (int k = r - 1; k >= 0; --k) {   // L^T w = z
            FF acc{0.f, 0.f};
            for (int l = k + 1 + lane; l < r; l += 32)
                acc = ff_fma_acc(acc, ld_ff(M + (size_t)l * r + k), ld_ff(sv + (int64_t)l * kSkNQ));
            acc = ff_warp_sum(acc);
            if (lane == 0) st_ff(sv + (int64_t)k * kSkNQ, ff_fms(ld_ff(sv + (int64_t)k * kSkNQ), acc, FF{1.f, 0.f}));
            __syncwarp();
        }
        for (int k = lane; k < r; k += 32) st_ff(cv + (int64_t)pv[k] * cst, ld_ff(sv + (int64_t)k * kSkNQ));
    } else if (lane < nq) {
        const int q = lane;
        for (int k = 0; k < r; ++k) {
            FF z = ld_ff(sv + (int64_t)k * kSkNQ + q);
            for (int l = 0; l < k; ++l) z = ff_fms(z, ld_ff(M + (size_t)l * r + k), ld_ff(sv + (int64_t)l * kSkNQ + q));
            st_ff(sv + (int64_t)k * kSkNQ + q, ff_mul(z, ld_ff(M + (size_t)k * r + k)));
        }
        for (int k = r - 1; k >= 0; --k) {
            FF z = ld_ff(sv + (int64_t)k * kSkNQ + q);
            for (int l = k + 1; l < r; ++l) z = ff_fms(z, ld_ff(M + (size_t)l * r + k), ld_ff(sv + (int64_t)l * kSkNQ + q));
            st_ff(sv + (int64_t)k * kSkNQ + q, z);
        }
        for (int k = 0; k < r; ++k) st_ff(cv + (int64_t)pv[k] * cst + q, ld_ff(sv + (int64_t)k * kSkNQ + q));
    }
}

// The pivot sums of the large blocks, one warp per (block, pivot) item, so that
// a few large blocks (the coarse levels) spread over the whole GPU instead of
// leaving one warp each running long after the rest:
//   TR = false: s_k = sum_{j in Y} K(sigma_k, p_j) x_j   (forward product)
//   TR = true:  u_k = sum_{i in X} K(p_i, tau_k) x_i     (transpose product)
// written to sbig in the layout the source-side kernels read.
template <class T, int NQ, bool FF_, bool TR>
__global__ void __launch_bounds__(kSkThreads) k_skel_rows(SkelArgs S, const int2 *__restrict__ items, int64_t nitems,
                                                          const T *__restrict__ xs, int nq) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (kSkThreads / 32);
    for (int64_t it = ((int64_t)blockIdx.x * kSkThreads + threadIdx.x) >> 5; it < nitems; it += nw) {
        const int2 I = items[it];
        const int64_t b = I.x, po = S.piv_off[b];
        const int k = I.y;
        int p, j0, j1;
        if (TR) {
            p = S.box_start[S.blk_src[b]] + S.tau[po + k];
            j0 = S.box_start[S.blk_tgt[b]];
            j1 = S.box_end[S.blk_tgt[b]];
        } else {
            p = S.box_start[S.blk_tgt[b]] + S.sigma[po + k];
            j0 = S.box_start[S.blk_src[b]];
            j1 = S.box_end[S.blk_src[b]];
        }
        double *out = S.sbig + (S.bigpo[b] + k) * kSkNQ;
        if constexpr (FF_) {
            const float4 ph = S.fh[p], pl = S.fl[p];
            FF fa[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) fa[q] = FF{0.f, 0.f};
            for (int j = j0 + lane; j < j1; j += 32) {
                const FF kv = TR ? ff_kernel(S.kind, S.fh[j], S.fl[j], ph, pl) : ff_kernel(S.kind, ph, pl, S.fh[j], S.fl[j]);
#pragma unroll
                for (int q = 0; q < NQ; ++q)
                    if (q < nq) fa[q] = ff_fma_acc(fa[q], kv, (float)xs[(int64_t)j * nq + q]);
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nq) {
                    const FF v = ff_warp_sum(fa[q]);
                    if (lane == 0) st_ff(out + q, v);
                }
        } else {
            double acc[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
            for (int j = j0 + lane; j < j1; j += 32) {
                const double kv = TR ? skel_k(S.kind, S.kappa, S.px, S.py, S.pz, j, p)
                                     : skel_k(S.kind, S.kappa, S.px, S.py, S.pz, p, j);
#pragma unroll
                for (int q = 0; q < NQ; ++q)
                    if (q < nq) acc[q] += kv * (double)xs[(int64_t)j * nq + q];
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nq) {
                    double v = acc[q];
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) out[q] = v;
                }
        }
    }
}

// FF_: entries, sums, solves and the solved coefficients in float-float (FP32
// handles, Laplace and 1/r^4); pivot sums and coefficients then occupy their
// double slots as float-float pairs.
template <class T, int NQ, bool FF_>
__global__ void __launch_bounds__(kSkThreads) k_skel_src(SkelArgs S, const T *__restrict__ xs, int nq) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * kSkThreads + threadIdx.x) >> 5;
    for (;;) {
        const int64_t b = skel_next_block(S, lane);
        if (b >= S.nblk) break;
        const int r = S.rank[b];
        if (r == 0) continue;
        const int X = S.blk_tgt[b], Y = S.blk_src[b];
        const int x0 = S.box_start[X], y0 = S.box_start[Y], y1 = S.box_end[Y];
        const int64_t po = S.piv_off[b];
        const int *sg = S.sigma + po;
        double *sv = S.sbuf + w0 * (int64_t)S.mr * kSkNQ, *cv = S.cbuf + po * S.cst;
        const double *M = S.lu + S.lu_off[b];
        const int *pv = S.lu_piv + po;
        const int64_t bp = S.bigpo[b];
        if (bp >= 0) sv = S.sbig + bp * kSkNQ;   // a large block: its sums are ready
        int kb = bp >= 0 ? r : 0;
        if (NQ == 1 && FF_ && kb == 0 && y1 - y0 <= 64) {
            // few source points (the leaf level): lane k sums pivot k over all of
            // them (the points are read by every lane at once), no warp sums
            for (int k = lane; k < r; k += 32) {
                const int ps = x0 + sg[k];
                const float4 ph = S.fh[ps], pl = S.fl[ps];
                FF a{0.f, 0.f};
                for (int j = y0; j < y1; ++j) a = ff_fma_acc(a, ff_kernel(S.kind, ph, pl, S.fh[j], S.fl[j]), (float)xs[j]);
                st_ff(sv + (int64_t)k * kSkNQ, a);
            }
            kb = r;
        }
        if (NQ == 1 && FF_)   // as below, entries and sums in float-float
            for (; kb + 4 <= r; kb += 4) {
                float4 ph[4], pl[4];
                FF a4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int ps = x0 + sg[kb + u];
                    ph[u] = S.fh[ps];
                    pl[u] = S.fl[ps];
                    a4[u] = FF{0.f, 0.f};
                }
                for (int j = y0 + lane; j < y1; j += 32) {
                    const float4 jh = S.fh[j], jl = S.fl[j];
                    const float xv = (float)xs[j];
#pragma unroll
                    for (int u = 0; u < 4; ++u) a4[u] = ff_fma_acc(a4[u], ff_kernel(S.kind, ph[u], pl[u], jh, jl), xv);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const FF v = ff_warp_sum(a4[u]);
                    if (lane == 0) st_ff(sv + (int64_t)(kb + u) * kSkNQ, v);
                }
            }
        if (NQ == 1 && !FF_)   // four pivots at a time: each source point is loaded once per four entries
            for (; kb + 4 <= r; kb += 4) {
                double sx[4], sy[4], sz[4], a4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int ps = x0 + sg[kb + u];
                    sx[u] = S.px[ps];
                    sy[u] = S.py[ps];
                    sz[u] = S.pz[ps];
                    a4[u] = 0.0;
                }
                for (int j = y0 + lane; j < y1; j += 32) {
                    const double jx = S.px[j], jy = S.py[j], jz = S.pz[j], xv = (double)xs[j];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        a4[u] += skel_kd(S.kind, S.kappa, sx[u] - jx, sy[u] - jy, sz[u] - jz) * xv;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    double v = a4[u];
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) sv[(int64_t)(kb + u) * kSkNQ] = v;
                }
            }
        for (int k = kb; k < r; ++k) {
            const int ps = x0 + sg[k];
            double acc[NQ];
            if constexpr (FF_) {
                const float4 ph = S.fh[ps], pl = S.fl[ps];
                FF fa[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) fa[q] = FF{0.f, 0.f};
                for (int j = y0 + lane; j < y1; j += 32) {
                    const FF kv = ff_kernel(S.kind, ph, pl, S.fh[j], S.fl[j]);
#pragma unroll
                    for (int q = 0; q < NQ; ++q)
                        if (q < nq) fa[q] = ff_fma_acc(fa[q], kv, (float)xs[(int64_t)j * nq + q]);
                }
#pragma unroll
                for (int q = 0; q < NQ; ++q)
                    if (q < nq) {
                        const FF v = ff_warp_sum(fa[q]);
                        if (lane == 0) st_ff(sv + (int64_t)k * kSkNQ + q, v);
                    }
                continue;
            } else {
#pragma unroll
                for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
                for (int j = y0 + lane; j < y1; j += 32) {
                    const double kv = skel_k(S.kind, S.kappa, S.px, S.py, S.pz, ps, j);
#pragma unroll
                    for (int q = 0; q < NQ; ++q)
                        if (q < nq) acc[q] += kv * (double)xs[(int64_t)j * nq + q];
                }
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                if (q < nq) {
                    double v = acc[q];
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) sv[(int64_t)k * kSkNQ + q] = v;
                }
            }
        }
        __syncwarp();
        if constexpr (FF_) {
            ff_solve<NQ>(M, pv, r, sv, cv, S.cst, nq, lane);
            __syncwarp();
            continue;
        }
        if (NQ == 1 && r <= 64) {   // one column, rank <= 64: lane k holds z_k and z_(k+32)
            // column-oriented substitutions: one FMA per lane and column instead of a
            // dot product and a five-step FP64 warp sum per row
            const int k0 = lane, k1 = lane + 32;
            double z0 = k0 < r ? sv[(int64_t)pv[k0] * kSkNQ] : 0.0, z1 = k1 < r ? sv[(int64_t)pv[k1] * kSkNQ] : 0.0;
            const double i0 = k0 < r ? 1.0 / M[(size_t)k0 * r + k0] : 0.0, i1 = k1 < r ? 1.0 / M[(size_t)k1 * r + k1] : 0.0;
            for (int l = 0; l < r; ++l) {   // L z = P s (unit lower)
                const double zl = __shfl_sync(0xffffffffu, l < 32 ? z0 : z1, l & 31);
                if (k0 > l && k0 < r) z0 = fma(-M[(size_t)k0 * r + l], zl, z0);
                if (k1 > l && k1 < r) z1 = fma(-M[(size_t)k1 * r + l], zl, z1);
            }
            for (int l = r - 1; l >= 0; --l) {   // U c = z
                if (lane == (l & 31)) {
                    if (l < 32) z0 *= i0;
                    else z1 *= i1;
                }
                const double cl = __shfl_sync(0xffffffffu, l < 32 ? z0 : z1, l & 31);
                if (k0 < l) z0 = fma(-M[(size_t)k0 * r + l], cl, z0);
                if (k1 < l) z1 = fma(-M[(size_t)k1 * r + l], cl, z1);
            }
            if (k0 < r) cv[(int64_t)k0 * S.cst] = z0;
            if (k1 < r) cv[(int64_t)k1 * S.cst] = z1;
        } else if (NQ == 1) {   // one column, larger rank: the warp shares each dot product
            for (int k = 0; k < r; ++k) {   // L z = P s (unit lower)
                double acc = 0.0;
                for (int l = lane; l < k; l += 32) acc += M[(size_t)k * r + l] * cv[(int64_t)l * S.cst];
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) cv[(int64_t)k * S.cst] = sv[(int64_t)pv[k] * kSkNQ] - acc;
                __syncwarp();
            }
            for (int k = r - 1; k >= 0; --k) {   // U c = z
                double acc = 0.0;
                for (int l = k + 1 + lane; l < r; l += 32) acc += M[(size_t)k * r + l] * cv[(int64_t)l * S.cst];
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) cv[(int64_t)k * S.cst] = (cv[(int64_t)k * S.cst] - acc) / M[(size_t)k * r + k];
                __syncwarp();
            }
        } else if (lane < nq) {   // lane q solves column q
            const int q = lane;
            for (int k = 0; k < r; ++k) {   // L z = P s (unit lower)
                double acc = 0.0;
                for (int l = 0; l < k; ++l) acc += M[(size_t)k * r + l] * cv[(int64_t)l * S.cst + q];
                cv[(int64_t)k * S.cst + q] = sv[(int64_t)pv[k] * kSkNQ + q] - acc;
            }
            for (int k = r - 1; k >= 0; --k) {   // U c = z
                double acc = 0.0;
                for (int l = k + 1; l < r; ++l) acc += M[(size_t)k * r + l] * cv[(int64_t)l * S.cst + q];
                cv[(int64_t)k * S.cst + q] = (cv[(int64_t)k * S.cst + q] - acc) / M[(size_t)k * r + k];
            }
        }
        __syncwarp();
    }
}

// per leaf: Y = near + sum over its ancestors' blocks of K(rows, tau) C.  The
// four warps split the blocks, lanes take rows (32 at a time); the partial sums
// are added in shared memory in warp order.  nearbuf is column-major (N x nq).
struct FFPivot {   // a staged pivot of the float-float path: coordinates, coefficient
    float4 h, l;
    float ch, cl;
};

template <class T, int NQ, bool FF_>
__global__ void __launch_bounds__(kSkThreads) k_skel_leaf(SkelArgs S, LeafArgs A, const int64_t *__restrict__ tgt_ptr,
                                                          const T *__restrict__ nearbuf, T *__restrict__ y, int64_t n,
                                                          int nq) {
    __shared__ double red[kSkThreads / 32][32][NQ];
    __shared__ Pt4d piv[kSkThreads / 32][NQ == 1 && !FF_ ? kSkLeafStage : 1];   // one column: a warp's staged pivots
    __shared__ FFPivot fpiv[kSkThreads / 32][NQ == 1 && FF_ ? kSkLeafStage : 1];
    const float2 *cff = reinterpret_cast<const float2 *>(S.cbuf);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int z = blockIdx.x;
    const int Zg = (int)(A.offL + z);
    const int zs = A.box_start[Zg], ze = A.box_end[Zg];
    for (int r0 = zs; r0 < ze; r0 += 32) {
        const int i = r0 + lane;
        const bool row = i < ze;
        double acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
        const double ix = row && !FF_ ? S.px[i] : 0.0, iy = row && !FF_ ? S.py[i] : 0.0,
                     iz = row && !FF_ ? S.pz[i] : 0.0;
        FF fa[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) fa[q] = FF{0.f, 0.f};
        const float4 fih = FF_ && row ? S.fh[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 fil = FF_ && row ? S.fl[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        int cnt = 0;
        for (int l = 1; l <= A.L; ++l) {
            const int Ag = A.leaf_anc[(int64_t)(l - 1) * A.nleaf + z];
            for (int64_t b = tgt_ptr[Ag]; b < tgt_ptr[Ag + 1]; ++b, ++cnt) {
                if ((cnt & 3) != warp) continue;
                const int r = S.rank[b];
                const int y0 = S.box_start[S.blk_src[b]];
                const int64_t po = S.piv_off[b];
                if constexpr (FF_) {
                    if (NQ == 1) {   // staged pivots, float-float entries and sums
                        for (int k0 = 0; k0 < r; k0 += kSkLeafStage) {
                            const int kn = min(kSkLeafStage, r - k0);
                            __syncwarp();
                            for (int k = lane; k < kn; k += 32) {
                                const int pt = y0 + S.tau[po + k0 + k];
                                const float2 c = cff[(po + k0 + k) * S.cst];
                                fpiv[warp][k] = FFPivot{S.fh[pt], S.fl[pt], c.x, c.y};
                            }
                            __syncwarp();
                            if (row)
                                for (int k = 0; k < kn; ++k) {
                                    const FFPivot p = fpiv[warp][k];
                                    fa[0] = ff_fma_acc(fa[0], ff_kernel(S.kind, fih, fil, p.h, p.l), FF{p.ch, p.cl});
                                }
                        }
                    } else {
                        for (int k = 0; k < r; ++k) {
                            const int pt = y0 + S.tau[po + k];
                            const FF kv = row ? ff_kernel(S.kind, fih, fil, S.fh[pt], S.fl[pt]) : FF{0.f, 0.f};
                            const float2 *cv = cff + (po + k) * S.cst;
#pragma unroll
                            for (int q = 0; q < NQ; ++q)
                                if (q < nq) {
                                    const float2 c = cv[q];
                                    fa[q] = ff_fma_acc(fa[q], kv, FF{c.x, c.y});
                                }
                        }
                    }
                    continue;
                }
                if (NQ == 1) {   // pivots (coordinates and coefficient) staged in shared memory
                    for (int k0 = 0; k0 < r; k0 += kSkLeafStage) {
                        const int kn = min(kSkLeafStage, r - k0);
                        __syncwarp();
                        for (int k = lane; k < kn; k += 32) {
                            const int pt = y0 + S.tau[po + k0 + k];
                            piv[warp][k] = make_pt4d(S.px[pt], S.py[pt], S.pz[pt], S.cbuf[(po + k0 + k) * S.cst]);
                        }
                        __syncwarp();
                        if (row)
                            for (int k = 0; k < kn; ++k) {
                                const Pt4d p = piv[warp][k];
                                acc[0] += skel_kd(S.kind, S.kappa, ix - p.x, iy - p.y, iz - p.z) * p.w;
                            }
                    }
                    continue;
                }
                for (int k = 0; k < r; ++k) {
                    const double kv = row ? skel_k(S.kind, S.kappa, S.px, S.py, S.pz, i, y0 + S.tau[po + k]) : 0.0;
                    const double *cv = S.cbuf + (po + k) * S.cst;
#pragma unroll
                    for (int q = 0; q < NQ; ++q)
                        if (q < nq) acc[q] += kv * cv[q];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) red[warp][lane][q] = FF_ ? ff_to_double(fa[q]) : acc[q];
        __syncthreads();
        if (warp == 0 && row) {
            const int64_t o = A.perm[i];
            for (int q = 0; q < nq; ++q) {
                const double v = ((red[0][lane][q] + red[1][lane][q]) + red[2][lane][q]) + red[3][lane][q];
                y[(int64_t)q * n + o] = (T)(v + (double)nearbuf[(int64_t)q * n + i]);
            }
        }
        __syncthreads();
    }
}

// transpose, per block (one warp): u = K(X,tau)^T X_X for the pass's columns,
// then a = M^{-T} u from P M = L U: U^T z = u, L^T w = z, a = P^T w.
template <class T, int NQ, bool FF_>
__global__ void __launch_bounds__(kSkThreads) k_skelT_src(SkelArgs S, const T *__restrict__ xs, int nq) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * kSkThreads + threadIdx.x) >> 5;
    for (;;) {
        const int64_t b = skel_next_block(S, lane);
        if (b >= S.nblk) break;
        const int r = S.rank[b];
        if (r == 0) continue;
        const int X = S.blk_tgt[b], Y = S.blk_src[b];
        const int x0 = S.box_start[X], x1 = S.box_end[X], y0 = S.box_start[Y];
        const int64_t po = S.piv_off[b];
        const int *ta = S.tau + po;
        double *sv = S.sbuf + w0 * (int64_t)S.mr * kSkNQ, *cv = S.cbuf + po * S.cst;
        const double *M = S.lu + S.lu_off[b];
        const int *pv = S.lu_piv + po;
        const int64_t bp = S.bigpo[b];
        if (bp >= 0) sv = S.sbig + bp * kSkNQ;   // a large block: its sums are ready
        int k0 = bp >= 0 ? r : 0;
        if (NQ == 1 && FF_ && k0 == 0 && x1 - x0 <= 64) {   // few target points: lane k takes pivot k
            for (int k = lane; k < r; k += 32) {
                const int pt = y0 + ta[k];
                const float4 ph = S.fh[pt], pl = S.fl[pt];
                FF a{0.f, 0.f};
                for (int i = x0; i < x1; ++i) a = ff_fma_acc(a, ff_kernel(S.kind, S.fh[i], S.fl[i], ph, pl), (float)xs[i]);
                st_ff(sv + (int64_t)k * kSkNQ, a);
            }
            k0 = r;
        }
        for (int k = k0; k < r; ++k) {
            const int pt = y0 + ta[k];
            double acc[NQ];
            if constexpr (FF_) {
                const float4 ph = S.fh[pt], pl = S.fl[pt];
                FF fa[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) fa[q] = FF{0.f, 0.f};
                for (int i = x0 + lane; i < x1; i += 32) {
                    const FF kv = ff_kernel(S.kind, S.fh[i], S.fl[i], ph, pl);
#pragma unroll
                    for (int q = 0; q < NQ; ++q)
                        if (q < nq) fa[q] = ff_fma_acc(fa[q], kv, (float)xs[(int64_t)i * nq + q]);
                }
#pragma unroll
                for (int q = 0; q < NQ; ++q)
                    if (q < nq) {
                        const FF v = ff_warp_sum(fa[q]);
                        if (lane == 0) st_ff(sv + (int64_t)k * kSkNQ + q, v);
                    }
                continue;
            } else {
#pragma unroll
                for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
                for (int i = x0 + lane; i < x1; i += 32) {
                    const double kv = skel_k(S.kind, S.kappa, S.px, S.py, S.pz, i, pt);
#pragma unroll
                    for (int q = 0; q < NQ; ++q)
                        if (q < nq) acc[q] += kv * (double)xs[(int64_t)i * nq + q];
                }
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                if (q < nq) {
                    double v = acc[q];
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) sv[(int64_t)k * kSkNQ + q] = v;
                }
            }
        }
        __syncwarp();
        if constexpr (FF_) {
            ff_solve_T<NQ>(M, pv, r, sv, cv, S.cst, nq, lane);
            __syncwarp();
            continue;
        }
        // z and w overwrite u in sv; a is scattered into cv by the row order
        if (NQ == 1 && r <= 64) {   // one column, rank <= 64: lane k holds entries k and k + 32
            const int k0 = lane, k1 = lane + 32;
            double z0 = k0 < r ? sv[(int64_t)k0 * kSkNQ] : 0.0, z1 = k1 < r ? sv[(int64_t)k1 * kSkNQ] : 0.0;
            const double i0 = k0 < r ? 1.0 / M[(size_t)k0 * r + k0] : 0.0, i1 = k1 < r ? 1.0 / M[(size_t)k1 * r + k1] : 0.0;
            for (int l = 0; l < r; ++l) {   // U^T z = u (column l of U^T is row l of U)
                if (lane == (l & 31)) {
                    if (l < 32) z0 *= i0;
                    else z1 *= i1;
                }
                const double zl = __shfl_sync(0xffffffffu, l < 32 ? z0 : z1, l & 31);
                if (k0 > l && k0 < r) z0 = fma(-M[(size_t)l * r + k0], zl, z0);
                if (k1 > l && k1 < r) z1 = fma(-M[(size_t)l * r + k1], zl, z1);
            }
            for (int l = r - 1; l >= 0; --l) {   // L^T w = z (unit diagonal)
                const double wl = __shfl_sync(0xffffffffu, l < 32 ? z0 : z1, l & 31);
                if (k0 < l) z0 = fma(-M[(size_t)l * r + k0], wl, z0);
                if (k1 < l) z1 = fma(-M[(size_t)l * r + k1], wl, z1);
            }
            if (k0 < r) cv[(int64_t)pv[k0] * S.cst] = z0;
            if (k1 < r) cv[(int64_t)pv[k1] * S.cst] = z1;
        } else if (NQ == 1) {
            for (int k = 0; k < r; ++k) {   // U^T z = u
                double acc = 0.0;
                for (int l = lane; l < k; l += 32) acc += M[(size_t)l * r + k] * sv[(int64_t)l * kSkNQ];
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) sv[(int64_t)k * kSkNQ] = (sv[(int64_t)k * kSkNQ] - acc) / M[(size_t)k * r + k];
                __syncwarp();
            }
            for (int k = r - 1; k >= 0; --k) {   // L^T w = z (unit diagonal)
                double acc = 0.0;
                for (int l = k + 1 + lane; l < r; l += 32) acc += M[(size_t)l * r + k] * sv[(int64_t)l * kSkNQ];
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) sv[(int64_t)k * kSkNQ] -= acc;
                __syncwarp();
            }
            for (int k = lane; k < r; k += 32) cv[(int64_t)pv[k] * S.cst] = sv[(int64_t)k * kSkNQ];
        } else if (lane < nq) {
            const int q = lane;
            for (int k = 0; k < r; ++k) {
                double acc = 0.0;
                for (int l = 0; l < k; ++l) acc += M[(size_t)l * r + k] * sv[(int64_t)l * kSkNQ + q];
                sv[(int64_t)k * kSkNQ + q] = (sv[(int64_t)k * kSkNQ + q] - acc) / M[(size_t)k * r + k];
            }
            for (int k = r - 1; k >= 0; --k) {
                double acc = 0.0;
                for (int l = k + 1; l < r; ++l) acc += M[(size_t)l * r + k] * sv[(int64_t)l * kSkNQ + q];
                sv[(int64_t)k * kSkNQ + q] -= acc;
            }
            for (int k = 0; k < r; ++k) cv[(int64_t)pv[k] * S.cst + q] = sv[(int64_t)k * kSkNQ + q];
        }
        __syncwarp();
    }
}

// transpose, per leaf: Y = near + sum over blocks whose source is an ancestor of
// the leaf of K(sigma, rows)^T a, blocks taken from the source-major index
template <class T, int NQ, bool FF_>
__global__ void __launch_bounds__(kSkThreads) k_skelT_leaf(SkelArgs S, LeafArgs A, const int64_t *__restrict__ src_ptr,
                                                           const int64_t *__restrict__ src_order,
                                                           const T *__restrict__ nearbuf, T *__restrict__ y,
                                                           int64_t n, int nq) {
    __shared__ double red[kSkThreads / 32][32][NQ];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int z = blockIdx.x;
    const int Zg = (int)(A.offL + z);
    const int zs = A.box_start[Zg], ze = A.box_end[Zg];
    for (int r0 = zs; r0 < ze; r0 += 32) {
        const int i = r0 + lane;
        const bool row = i < ze;
        double acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
        FF fa[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) fa[q] = FF{0.f, 0.f};
        const float4 fih = FF_ && row ? S.fh[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 fil = FF_ && row ? S.fl[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 *cff = reinterpret_cast<const float2 *>(S.cbuf);
        int cnt = 0;
        for (int l = 1; l <= A.L; ++l) {
            const int Bg = A.leaf_anc[(int64_t)(l - 1) * A.nleaf + z];
            for (int64_t e = src_ptr[Bg]; e < src_ptr[Bg + 1]; ++e, ++cnt) {
                if ((cnt & 3) != warp) continue;
                const int64_t b = src_order[e];
                const int r = S.rank[b];
                const int x0 = S.box_start[S.blk_tgt[b]];
                const int64_t po = S.piv_off[b];
                if constexpr (FF_) {
                    for (int k = 0; k < r; ++k) {
                        const int pt = x0 + S.sigma[po + k];
                        const FF kv = row ? ff_kernel(S.kind, S.fh[pt], S.fl[pt], fih, fil) : FF{0.f, 0.f};
                        const float2 *cv = cff + (po + k) * S.cst;
#pragma unroll
                        for (int q = 0; q < NQ; ++q)
                            if (q < nq) {
                                const float2 c = cv[q];
                                fa[q] = ff_fma_acc(fa[q], kv, FF{c.x, c.y});
                            }
                    }
                    continue;
                }
                for (int k = 0; k < r; ++k) {
                    const double kv = row ? skel_k(S.kind, S.kappa, S.px, S.py, S.pz, x0 + S.sigma[po + k], i) : 0.0;
                    const double *cv = S.cbuf + (po + k) * S.cst;
#pragma unroll
                    for (int q = 0; q < NQ; ++q)
                        if (q < nq) acc[q] += kv * cv[q];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) red[warp][lane][q] = FF_ ? ff_to_double(fa[q]) : acc[q];
        __syncthreads();
        if (warp == 0 && row) {
            const int64_t o = A.perm[i];
            for (int q = 0; q < nq; ++q) {
                const double v = ((red[0][lane][q] + red[1][lane][q]) + red[2][lane][q]) + red[3][lane][q];
                y[(int64_t)q * n + o] = (T)(v + (double)nearbuf[(int64_t)q * n + i]);
            }
        }
        __syncthreads();
    }
}

// float-float offsets of the sorted points from the domain centre c0: the high
// part is the FP32 rounding of the FP64 offset, the low part the FP32 rounding
// of the remainder (together within 2^-48 of the offset)
__global__ void k_ff_coords(const double *__restrict__ px, const double *__restrict__ py,
                            const double *__restrict__ pz, double c0x, double c0y, double c0z, int64_t n,
                            float4 *__restrict__ hi, float4 *__restrict__ lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const FF x = ff_from_double(px[i] - c0x), y = ff_from_double(py[i] - c0y), z = ff_from_double(pz[i] - c0z);
    hi[i] = make_float4(x.h, y.h, z.h, 0.f);
    lo[i] = make_float4(x.l, y.l, z.l, 0.f);
}

SkelArgs skel_args(Handle &h) {
    SkelArgs S{};
    S.kind = h.kernel;
    S.kappa = h.kappa;
    S.px = h.px; S.py = h.py; S.pz = h.pz;
    S.fh = h.sffh; S.fl = h.sffl;
    S.nblk = h.nblk;
    S.blk_tgt = h.blk_tgt; S.blk_src = h.blk_src; S.box_start = h.box_start; S.box_end = h.box_end;
    S.rank = h.rank; S.sigma = h.sigma; S.tau = h.tau;
    S.piv_off = h.piv_off; S.lu_off = h.lu_off;
    S.lu = h.lu; S.lu_piv = h.lu_piv;
    S.sbuf = h.skel_s; S.cbuf = h.skel_c;
    S.mr = std::max(1, h.max_rank);
    S.cst = std::max(1, h.skel_nq);
    S.next = h.skel_next;
    S.ff = h.sffh != nullptr;
    S.bigpo = h.skel_bigpo;
    S.sbig = h.skel_sbig;
    return S;
}

int skel_src_grid(const Handle &h) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((h.nblk * 32 + kSkThreads - 1) / kSkThreads, 16LL * num_sms()));
}

// the source-side and leaf kernels of one pass
template <class T, bool FF_>
void skel_launch(Handle &h, const SkelArgs &S, const LeafArgs &A, const T *xs, const T *nearbuf, T *yq, int nq,
                 bool transpose, cudaStream_t s) {
    const int64_t n = h.N;
    if (h.nblk > 0) {
        const int grid = skel_src_grid(h);
        if (h.skel_nbig > 0) {   // pivot sums of the large blocks first
            const int rg = (int)std::min<int64_t>((h.skel_nbig * 32 + kSkThreads - 1) / kSkThreads, 16LL * num_sms());
            if (transpose) {
                if (nq == 1) k_skel_rows<T, 1, FF_, true><<<rg, kSkThreads, 0, s>>>(S, h.skel_big, h.skel_nbig, xs, nq);
                else k_skel_rows<T, kSkNQ, FF_, true><<<rg, kSkThreads, 0, s>>>(S, h.skel_big, h.skel_nbig, xs, nq);
            } else {
                if (nq == 1) k_skel_rows<T, 1, FF_, false><<<rg, kSkThreads, 0, s>>>(S, h.skel_big, h.skel_nbig, xs, nq);
                else k_skel_rows<T, kSkNQ, FF_, false><<<rg, kSkThreads, 0, s>>>(S, h.skel_big, h.skel_nbig, xs, nq);
            }
        }
        H3D_CUDA(cudaMemsetAsync(h.skel_next, 0, sizeof(int), s));
        if (transpose) {
            if (nq == 1) k_skelT_src<T, 1, FF_><<<grid, kSkThreads, 0, s>>>(S, xs, nq);
            else k_skelT_src<T, kSkNQ, FF_><<<grid, kSkThreads, 0, s>>>(S, xs, nq);
        } else {
            if (nq == 1) k_skel_src<T, 1, FF_><<<grid, kSkThreads, 0, s>>>(S, xs, nq);
            else k_skel_src<T, kSkNQ, FF_><<<grid, kSkThreads, 0, s>>>(S, xs, nq);
        }
    }
    if (transpose) {
        if (nq == 1)
            k_skelT_leaf<T, 1, FF_><<<h.nleaf, kSkThreads, 0, s>>>(S, A, h.skel_src_ptr, h.skel_src_order, nearbuf, yq, n,
                                                                  nq);
        else
            k_skelT_leaf<T, kSkNQ, FF_><<<h.nleaf, kSkThreads, 0, s>>>(S, A, h.skel_src_ptr, h.skel_src_order, nearbuf,
                                                                      yq, n, nq);
    } else {
        if (nq == 1) k_skel_leaf<T, 1, FF_><<<h.nleaf, kSkThreads, 0, s>>>(S, A, h.tgt_ptr, nearbuf, yq, n, nq);
        else k_skel_leaf<T, kSkNQ, FF_><<<h.nleaf, kSkThreads, 0, s>>>(S, A, h.tgt_ptr, nearbuf, yq, n, nq);
    }
}

// nearbuf[(q0 + q) n + i] = nmr[i kNQ + q], q < qn: a block of the multi-column
// near field (point-major) into the skeleton pass's column-major near buffer
template <class T>
__global__ void k_mr_to_cols(const T *__restrict__ nmr, int64_t n, int q0, int qn, T *__restrict__ nearbuf) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * qn) return;
    const int64_t i = e / qn;
    const int q = (int)(e - i * qn);
    nearbuf[(int64_t)(q0 + q) * n + i] = nmr[i * kNQ + q];
}

// one pass of up to kSkNQ columns: x, y column-major (N x nrhs), from column q0;
// FF_: float-float entries (FP32 handles of a kernel float-float evaluates)
template <class T, bool FF_>
void matvec_skel_pass(Handle &h, const T *x, T *y, int q0, int nq, bool transpose, cudaStream_t s) {
    const int64_t n = h.N;
    T *xs = (T *)h.skel_xs, *nearbuf = (T *)h.skel_near, *x1 = (T *)h.xs;
    LeafArgs A = leaf_args(h);
    k_skel_permute<T><<<gridn(n * nq, 256), 256, 0, s>>>(x, n, q0, nq, h.perm, xs);
    // near field on the side stream: blocks of kNQ columns through the multi-column
    // kernel where the leaves fit it, else one column at a time
    const int near_grid = sizeof(T) == 4 ? std::min(h.nleaf, kNearCtasPerSm * num_sms()) : h.nleaf;
    const bool near8 = nq > 1 && h.skel_xmr;
    for (int q = 0; near8 && q < nq; q += kNQ) {
        const int qn = std::min(kNQ, nq - q);
        k_permute_in_mr<T><<<gridn(n, 256), 256, 0, s>>>(x, n, q0 + q, qn, h.perm, (T *)h.skel_xmr);
        H3D_CUDA(cudaEventRecord(h.ev_fork, s));
        H3D_CUDA(cudaStreamWaitEvent(h.side_stream, h.ev_fork, 0));
        k_near_mr<T><<<h.nleaf, kLeafThreads, 0, h.side_stream>>>(A, (const T *)h.skel_xmr, (T *)h.skel_nmr);
        k_mr_to_cols<T><<<gridn(n * qn, 256), 256, 0, h.side_stream>>>((const T *)h.skel_nmr, n, q, qn,
                                                                       nearbuf);
        H3D_CUDA(cudaEventRecord(h.ev_join, h.side_stream));
        H3D_CUDA(cudaStreamWaitEvent(s, h.ev_join, 0));   // the buffers are reused by the next block
    }
    for (int q = 0; !near8 && q < nq; ++q) {
        k_permute_in<T><<<gridn(n, 256), 256, 0, s>>>(x + (size_t)(q0 + q) * n, h.perm, n, x1);
        H3D_CUDA(cudaEventRecord(h.ev_fork, s));
        H3D_CUDA(cudaStreamWaitEvent(h.side_stream, h.ev_fork, 0));
        k_near<T><<<near_grid, kLeafThreads, 0, h.side_stream>>>(A, x1, nearbuf + (size_t)q * n);
        H3D_CUDA(cudaEventRecord(h.ev_join, h.side_stream));
        H3D_CUDA(cudaStreamWaitEvent(s, h.ev_join, 0));   // x1 is reused by the next column
    }
    SkelArgs S = skel_args(h);
    T *yq = y + (size_t)q0 * n;
    skel_launch<T, FF_>(h, S, A, xs, nearbuf, yq, nq, transpose, s);
    H3D_LAUNCH_CHECK();
}

}  // namespace

void build_matvec_plan(Handle &h, cudaStream_t s, Arena &tmp) {
    (void)tmp;
    H3D_CUDA(cudaFuncSetAttribute(k_leaf<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeafDynSmem));
    H3D_CUDA(cudaFuncSetAttribute(k_leaf<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeafDynSmem));
    H3D_CUDA(cudaFuncSetAttribute(k_leaf_mr<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeafDynSmem));
    H3D_CUDA(cudaFuncSetAttribute(k_leaf_mr<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeafDynSmem));
    H3D_CUDA(cudaFuncSetAttribute(k_tc_stream<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTsDynSmem));
    H3D_CUDA(cudaFuncSetAttribute(k_tc_stream<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTsDynSmem));
    H3D_CUDA(cudaFuncSetAttribute(k_tc_stream<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    H3D_CUDA(cudaFuncSetAttribute(k_tc_stream<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
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
    // the 32-column path's own row tasks (tall: kTaskRowsW rows) and splits
    std::vector<int4> wtasks;
    std::vector<int64_t> wpbase, wspbase;
    std::vector<int> wsbox, wsntask;
    int64_t pelw = 0;
    for (int64_t g = 0; g < nboxes; ++g) {
        if (Rv[g] == 0) continue;
        const int n = be[g] - bs[g];
        const int nt = (n + kTaskRowsW - 1) / kTaskRowsW;
        if (nt == 1) {
            wtasks.push_back(make_int4((int)g, 0, n, 1));
            wpbase.push_back(-1);
        } else {
            const int per = (n + nt - 1) / nt;
            wsbox.push_back((int)g);
            wsntask.push_back(nt);
            wspbase.push_back(pelw);
            for (int k = 0; k < nt; ++k) {
                wtasks.push_back(make_int4((int)g, k * per, std::min(n, (k + 1) * per), 0));
                wpbase.push_back(pelw + (int64_t)k * ldv[g]);
            }
            pelw += (int64_t)nt * ldv[g];
            h.max_rv_split_w = std::max(h.max_rv_split_w, Rv[g]);
        }
    }
    h.nsplit_w = (int)wsbox.size();
    h.split_box_w = h.mem.get<int>(std::max<size_t>(wsbox.size(), 1));
    h.split_ntask_w = h.mem.get<int>(std::max<size_t>(wsbox.size(), 1));
    h.split_pbase_w = h.mem.get<int64_t>(std::max<size_t>(wsbox.size(), 1));
    if (!wsbox.empty()) {
        H3D_CUDA(cudaMemcpyAsync(h.split_box_w, wsbox.data(), wsbox.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        H3D_CUDA(cudaMemcpyAsync(h.split_ntask_w, wsntask.data(), wsbox.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        H3D_CUDA(cudaMemcpyAsync(h.split_pbase_w, wspbase.data(), wsbox.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                 s));
    }
    h.partial_elems_w = pelw;
    // tensor-core gather work items: (wide task, block of kTcCols columns), resolved,
    // and one 2-D tensor map per source box (FP32 handles whose leaves fit the
    // 32-column path only)
    {
        std::vector<int64_t> vb(nboxes);
        H3D_CUDA(cudaMemcpyAsync(vb.data(), h.vbase, nboxes * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        std::vector<int64_t> vc0(nboxes);
        H3D_CUDA(cudaMemcpyAsync(vc0.data(), h.vcol0, nboxes * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        H3D_CUDA(cudaStreamSynchronize(s));
        const bool wide = h.prec == H3D_FP32 && h.tf32 && h.leaf_size <= kMaxLeafW && h.storage == H3D_STORE_FACTORS;
        std::vector<int> tmap_of(nboxes, -1);
        std::vector<CUtensorMap> tmaps;
        if (wide) {
            void *fn = nullptr;
            cudaDriverEntryPointQueryResult q{};
            H3D_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
            if (!fn || q != cudaDriverEntryPointSuccess) throw Error{H3D_ERR_CUDA};   // driver without tensor maps
            auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
            for (int64_t g = 0; g < nboxes; ++g) {
                if (Rv[g] == 0) continue;
                CUtensorMap tm;
                const cuuint64_t dims[2] = {(cuuint64_t)ldv[g], (cuuint64_t)(be[g] - bs[g])};
                const cuuint64_t strides[1] = {(cuuint64_t)ldv[g] * sizeof(float)};
                const cuuint32_t box[2] = {(cuuint32_t)kTcCols, (cuuint32_t)kTsK};
                const cuuint32_t estr[2] = {1, 1};
                const CUresult r = encode(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (float *)h.V + vb[g], dims, strides,
                                          box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS) throw Error{H3D_ERR_CUDA};
                tmap_of[g] = (int)tmaps.size();
                tmaps.push_back(tm);
            }
        }
        h.tc_tmaps = h.mem.get<unsigned char>(std::max<size_t>(tmaps.size(), 1) * sizeof(CUtensorMap));
        if (!tmaps.empty())
            H3D_CUDA(cudaMemcpyAsync(h.tc_tmaps, tmaps.data(), tmaps.size() * sizeof(CUtensorMap),
                                     cudaMemcpyHostToDevice, s));
        std::vector<TcGatherItem> items;
        for (size_t q = 0; wide && q < wtasks.size(); ++q) {
            const int Y = wtasks[q].x;
            const int nb = (Rv[Y] + kTcCols - 1) / kTcCols;
            for (int cb = 0; cb < nb; ++cb) {
                const int c_lo = cb * kTcCols;
                TcGatherItem g{};
                g.x = (int64_t)bs[Y] + wtasks[q].y;
                g.to_t = wtasks[q].w;
                g.o = g.to_t ? vc0[Y] + c_lo : wpbase[q] + c_lo;
                g.tmap = tmap_of[Y];
                g.c_lo = c_lo;
                g.r0 = wtasks[q].y;
                g.nrows = wtasks[q].z - wtasks[q].y;
                g.ncols = std::min(kTcCols, Rv[Y] - c_lo);
                items.push_back(g);
            }
        }
        h.ntc_items = (int)items.size();
        h.tc_items = h.mem.get<TcGatherItem>(std::max<size_t>(items.size(), 1));
        if (!items.empty())
            H3D_CUDA(cudaMemcpyAsync(h.tc_items, items.data(), items.size() * sizeof(TcGatherItem),
                                     cudaMemcpyHostToDevice, s));
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
    // the skeleton storage's products use none of the factor-streaming scratch
    const bool stream = h.storage != H3D_STORE_SKELETON;
    h.partial = h.mem.alloc((size_t)std::max<int64_t>(stream ? pel : 0, 4) * es);
    h.t = h.mem.alloc((size_t)std::max<int64_t>(stream ? h.sum_rank : 0, 4) * es);
    h.xs = h.mem.alloc((size_t)std::max<int64_t>(h.N, 4) * es);
    h.nearbuf = h.mem.alloc((size_t)std::max<int64_t>(h.N, 4) * es);
    if (stream && h.leaf_size <= kMaxLeafMR) {   // scratch of the multi-RHS product (kNQ columns per pass)
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
    if (h.symmetric()) {
        H3D_CUDA(cudaStreamCreateWithFlags(&h.sym_stream, cudaStreamNonBlocking));
        H3D_CUDA(cudaEventCreateWithFlags(&h.ev_sym_fork, cudaEventDisableTiming));
        H3D_CUDA(cudaEventCreateWithFlags(&h.ev_sym_join, cudaEventDisableTiming));
    }

    // transpose partials: per level l < L, per leaf z, R of its ancestor
    const int L = h.L, nleaf = h.nleaf;
    std::vector<int> anc((size_t)std::max(1, L) * nleaf);
    if (L > 0)
        H3D_CUDA(cudaMemcpyAsync(anc.data(), h.leaf_anc, anc.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
    H3D_CUDA(cudaStreamSynchronize(s));
    {   // far-field tiles: consecutive sibling leaves whose rows fit in 128
        std::vector<int> lld(nleaf);
        H3D_CUDA(cudaMemcpyAsync(lld.data(), h.leaf_ld, nleaf * sizeof(int), cudaMemcpyDeviceToHost, s));
        H3D_CUDA(cudaStreamSynchronize(s));
        std::vector<int2> tiles;
        for (int z = 0; z < nleaf;) {
            const int parent = L >= 2 ? anc[(size_t)(L - 2) * nleaf + z] : 0;
            int nl = 1, rows = lld[z];
            while (z + nl < nleaf && nl < kTileLeaves && rows + lld[z + nl] <= 128 &&
                   (L >= 2 ? anc[(size_t)(L - 2) * nleaf + z + nl] : 0) == parent) {
                rows += lld[z + nl];
                ++nl;
            }
            tiles.push_back(make_int2(z, nl));
            z += nl;
        }
        h.ntc_tiles = (int)tiles.size();
        h.tc_tiles = h.mem.get<int2>(std::max<size_t>(tiles.size(), 1));
        H3D_CUDA(cudaMemcpyAsync(h.tc_tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    }
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
    h.tpartial = h.mem.alloc((size_t)std::max<int64_t>(stream ? tel : 0, 4) * es);
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
    if (h.symmetric()) transpose = false;   // the operator is symmetric
    if (use_wide(h, nrhs, transpose)) return (nrhs + kNQW - 1) / kNQW;
    if (nrhs > 1 && !transpose && h.leaf_size <= kMaxLeafMR) return (nrhs + kNQ - 1) / kNQ;
    return nrhs;
}

void build_skeleton(Handle &h, cudaStream_t s, Arena &tmp) {
    const int64_t nblk = h.nblk;
    std::vector<int> rk(nblk);
    if (nblk > 0) H3D_CUDA(cudaMemcpyAsync(rk.data(), h.rank, nblk * sizeof(int), cudaMemcpyDeviceToHost, s));
    H3D_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> off(nblk + 1, 0);
    for (int64_t b = 0; b < nblk; ++b) off[b + 1] = off[b] + (int64_t)rk[b] * rk[b];
    h.lu_off_total = off[nblk];
    h.lu_off = h.mem.get<int64_t>((size_t)nblk + 1);
    H3D_CUDA(cudaMemcpyAsync(h.lu_off, off.data(), (nblk + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    h.lu = h.mem.get<double>((size_t)std::max<int64_t>(h.lu_off_total, 1));
    h.lu_piv = h.mem.get<int>((size_t)std::max<int64_t>(h.sum_rank, 1));
    // columns per pass: 16 unless the per-pivot solutions (FP64, sum_rank x columns)
    // would take more than a third of the memory left after the LU factors
    {
        size_t free_b = 0, total_b = 0;
        H3D_CUDA(cudaMemGetInfo(&free_b, &total_b));
        const double avail = (double)free_b - (double)h.lu_off_total * 8.0;
        h.skel_nq = kSkNQ;
        while (h.skel_nq > 1 && (double)h.sum_rank * h.skel_nq * 8.0 > avail / 3.0) h.skel_nq /= 2;
    }
    h.skel_s = h.mem.get<double>((size_t)skel_src_grid(h) * (kSkThreads / 32) * std::max(1, h.max_rank) * kSkNQ);
    {   // large blocks (r x max(m, n) >= kSkBig entries): one item per pivot
        std::vector<int> tg(nblk), sc(nblk), bs(h.n_boxes), be(h.n_boxes);
        if (nblk > 0) {
            H3D_CUDA(cudaMemcpyAsync(tg.data(), h.blk_tgt, nblk * sizeof(int), cudaMemcpyDeviceToHost, s));
            H3D_CUDA(cudaMemcpyAsync(sc.data(), h.blk_src, nblk * sizeof(int), cudaMemcpyDeviceToHost, s));
        }
        H3D_CUDA(cudaMemcpyAsync(bs.data(), h.box_start, h.n_boxes * sizeof(int), cudaMemcpyDeviceToHost, s));
        H3D_CUDA(cudaMemcpyAsync(be.data(), h.box_end, h.n_boxes * sizeof(int), cudaMemcpyDeviceToHost, s));
        H3D_CUDA(cudaStreamSynchronize(s));
        std::vector<int64_t> bigpo(std::max<int64_t>(nblk, 1), -1);
        std::vector<int2> items;
        int64_t slots = 0;
        for (int64_t b = 0; b < nblk; ++b) {
            const int64_t ext = std::max(be[tg[b]] - bs[tg[b]], be[sc[b]] - bs[sc[b]]);
            if ((int64_t)rk[b] * ext < kSkBig) continue;
            bigpo[b] = slots;
            for (int k = 0; k < rk[b]; ++k) items.push_back(make_int2((int)b, k));
            slots += rk[b];
        }
        h.skel_nbig = (int64_t)items.size();
        h.skel_bigpo = h.mem.get<int64_t>(bigpo.size());
        H3D_CUDA(cudaMemcpyAsync(h.skel_bigpo, bigpo.data(), bigpo.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        h.skel_big = h.mem.get<int2>(std::max<size_t>(items.size(), 1));
        if (!items.empty())
            H3D_CUDA(cudaMemcpyAsync(h.skel_big, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
        h.skel_sbig = h.mem.get<double>((size_t)std::max<int64_t>(slots, 1) * kSkNQ);
        H3D_CUDA(cudaStreamSynchronize(s));
    }
    h.skel_next = h.mem.get<int>(1);
    h.skel_c = h.mem.get<double>((size_t)std::max<int64_t>(h.sum_rank, 1) * h.skel_nq);
    if (h.prec == H3D_FP32 && ff_kernel_supported(h.kernel)) {   // float-float entries in the products
        h.sffh = h.mem.get<float4>((size_t)std::max<int64_t>(h.N, 1));
        h.sffl = h.mem.get<float4>((size_t)std::max<int64_t>(h.N, 1));
    }
    h.skel_xs = h.mem.alloc((size_t)std::max<int64_t>(h.N, 4) * kSkNQ * h.elem());
    if (h.leaf_size <= kMaxLeafMR) {   // multi-column near field of the passes (blocks of kNQ columns)
        h.skel_xmr = h.mem.alloc((size_t)std::max<int64_t>(h.N, 4) * kNQ * h.elem());
        h.skel_nmr = h.mem.alloc((size_t)std::max<int64_t>(h.N, 4) * kNQ * h.elem());
    }
    h.skel_near = h.mem.alloc((size_t)std::max<int64_t>(h.N, 4) * kSkNQ * h.elem());
    {   // blocks grouped by source box (stable), for the transpose product
        const int64_t nboxes = h.n_boxes;
        std::vector<int> src(nblk);
        if (nblk > 0) H3D_CUDA(cudaMemcpyAsync(src.data(), h.blk_src, nblk * sizeof(int), cudaMemcpyDeviceToHost, s));
        H3D_CUDA(cudaStreamSynchronize(s));
        std::vector<int64_t> ptr(nboxes + 1, 0), order(std::max<int64_t>(nblk, 1), 0);
        for (int64_t b = 0; b < nblk; ++b) ptr[src[b] + 1]++;
        for (int64_t g = 0; g < nboxes; ++g) ptr[g + 1] += ptr[g];
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t b = 0; b < nblk; ++b) order[fill[src[b]]++] = b;
        h.skel_src_ptr = h.mem.get<int64_t>((size_t)nboxes + 1);
        h.skel_src_order = h.mem.get<int64_t>(order.size());
        H3D_CUDA(cudaMemcpyAsync(h.skel_src_ptr, ptr.data(), ptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        H3D_CUDA(cudaMemcpyAsync(h.skel_src_order, order.data(), order.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                 s));
    }
    refactor_skeleton(h, s);
    H3D_CUDA(cudaStreamSynchronize(s));
    (void)tmp;
}

void refactor_skeleton(Handle &h, cudaStream_t s) {
    if (h.sffh) {
        const double c0[3] = {h.lo[0] + 0.5 * h.side, h.lo[1] + 0.5 * h.side, h.lo[2] + 0.5 * h.side};
        k_ff_coords<<<gridn(h.N, 256), 256, 0, s>>>(h.px, h.py, h.pz, c0[0], c0[1], c0[2], h.N, h.sffh, h.sffl);
        H3D_LAUNCH_CHECK();
    }
    if (h.nblk > 0) {
        SkelArgs S = skel_args(h);
        const int grid = (int)std::min<int64_t>(h.nblk, 4LL * num_sms());
        k_skel_factor<<<grid, kSkThreads, 0, s>>>(S);
        H3D_LAUNCH_CHECK();
    }
}

void matvec_skeleton(Handle &h, const void *x, void *y, int nrhs, bool transpose, cudaStream_t s) {
    const int width = std::max(1, std::min(kSkNQ, h.skel_nq));
    for (int q0 = 0; q0 < nrhs; q0 += width) {
        const int nq = std::min(width, nrhs - q0);
        if (h.prec == H3D_FP64)
            matvec_skel_pass<double, false>(h, (const double *)x, (double *)y, q0, nq, transpose, s);
        else if (h.sffh)
            matvec_skel_pass<float, true>(h, (const float *)x, (float *)y, q0, nq, transpose, s);
        else
            matvec_skel_pass<float, false>(h, (const float *)x, (float *)y, q0, nq, transpose, s);
    }
}

void run_matvec(Handle &h, const void *x, void *y, int nrhs, bool transpose, cudaStream_t s, cudaEvent_t *ev) {
    const int64_t n = h.N;
    if (h.storage == H3D_STORE_SKELETON) {
        matvec_skeleton(h, x, y, nrhs, transpose, s);
        return;
    }
    if (h.symmetric()) transpose = false;   // the operator is symmetric: A~^T = A~
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
