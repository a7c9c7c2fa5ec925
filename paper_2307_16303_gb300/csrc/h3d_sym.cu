// h3d_sym.cu -- products of symmetric storage (H3D_STORE_SYMMETRIC): the pairs
// whose factors are kept once ("fused" pairs).
//
// Every kernel here is symmetric, K(Y,X) = K(X,Y)^T, so the admissible blocks
// (X, Y) and (Y, X) of Alg. 2 share one approximation K(X,Y) ~ U V^T (Eq. prank;
// its transpose V U^T).  A fused pair is streamed from HBM once per product and
// serves both directions:
//   t  = V^T x_Y,   t' = U^T x_X,   y_X += U t,   y_Y += V t'.
// The pair's factors (U then V, column-major, leading dimensions = 2 mod 4) come into
// shared memory by one bulk copy per group of pairs, double-buffered, in a
// persistent grid of one CTA per SM.  A group of small pairs (the leaf level)
// is taken one pair per warp; a larger pair (the level above) by the whole CTA.
// Both directions add into an FP64 accumulator with atomic additions (each
// output row receives the contributions of all pairs it belongs to); after the
// near field is done the accumulator is added to the near-field buffer, which
// the leaf kernel then adds to the other pairs' far field.  The kernel runs on a
// stream of its own, beside the other pairs' gather: it is bound by latency
// (one CTA of 16 warps per SM) and leaves most of the HBM bandwidth to it.
//
// Sums: FP32 products are accumulated with fused multiply-adds in runs of four
// or eight terms (one column: packed two-lane FP32 FMAs over pairs of rows),
// each run added with Kahan compensation (FP64 handles: plain FP64).
#include "h3d_async.cuh"
#include "h3d_internal.cuh"

namespace h3d {

namespace {

struct SymArgs {
    const SymBlk *blk;
    const SymGroup *grp;
    int ngrp;
    int stage;                 // bytes per stage
    const unsigned char *F;    // symF
    int *err;                  // device-visible error word (a copy that did not arrive)
};

template <class T> struct KSum;
template <> struct KSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ float get() const { return s - c; }
};
template <> struct KSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double get() const { return s; }
};

// the NQ values of point i (point-major, i * NQ + q)
template <class T, int NQ>
__device__ __forceinline__ void load_x(const T *__restrict__ xs, int64_t i, T (&o)[NQ]) {
    if constexpr (NQ == 8 && sizeof(T) == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(xs + i * 8));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(xs + i * 8) + 1);
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
    } else if constexpr (NQ == 8) {
        const double2 *p = reinterpret_cast<const double2 *>(xs + i * 8);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const double2 v = __ldg(p + h);
            o[2 * h] = v.x;
            o[2 * h + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < NQ; ++q) o[q] = __ldg(xs + i * NQ + q);
    }
}

// the NQ coefficients of column k (shared memory, k * NQ + q)
template <class T, int NQ>
__device__ __forceinline__ void load_t(const T *t, int k, T (&o)[NQ]) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) o[q] = t[k * NQ + q];
}

// sum over l < len of c[l] x(x0 + l) for the NQ columns of x, in runs of four
// fused multiply-adds
template <class T, int NQ>
__device__ __forceinline__ void dot_x(const T *c, int len, const T *__restrict__ xs, int64_t x0, KSum<T> (&a)[NQ]) {
    int l = 0;
    for (; l + 4 <= len; l += 4) {
        T p[NQ], x[NQ];
        load_x<T, NQ>(xs, x0 + l, x);
        const T c0 = c[l];
#pragma unroll
        for (int q = 0; q < NQ; ++q) p[q] = c0 * x[q];
#pragma unroll
        for (int e = 1; e < 4; ++e) {
            load_x<T, NQ>(xs, x0 + l + e, x);
            const T ce = c[l + e];
#pragma unroll
            for (int q = 0; q < NQ; ++q) p[q] = fma(ce, x[q], p[q]);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) a[q].add(p[q]);
    }
    for (; l < len; ++l) {
        T x[NQ];
        load_x<T, NQ>(xs, x0 + l, x);
        const T cl = c[l];
#pragma unroll
        for (int q = 0; q < NQ; ++q) a[q].add(cl * x[q]);
    }
}

// sum over k < r of row[k * ld] t(k) for the NQ coefficient columns, in runs of four
template <class T, int NQ>
__device__ __forceinline__ void dot_t(const T *row, int ld, int r, const T *t, KSum<T> (&a)[NQ]) {
    int k = 0;
    for (; k + 4 <= r; k += 4) {
        T p[NQ], tv[NQ];
        load_t<T, NQ>(t, k, tv);
        const T u0 = row[k * ld];
#pragma unroll
        for (int q = 0; q < NQ; ++q) p[q] = u0 * tv[q];
#pragma unroll
        for (int e = 1; e < 4; ++e) {
            load_t<T, NQ>(t, k + e, tv);
            const T ue = row[(k + e) * ld];
#pragma unroll
            for (int q = 0; q < NQ; ++q) p[q] = fma(ue, tv[q], p[q]);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) a[q].add(p[q]);
    }
    for (; k < r; ++k) {
        T tv[NQ];
        load_t<T, NQ>(t, k, tv);
        const T uk = row[k * ld];
#pragma unroll
        for (int q = 0; q < NQ; ++q) a[q].add(uk * tv[q]);
    }
}

// One column (NQ = 1): two dot products at once, each in runs of eight terms
// split over two fused multiply-add chains, so that a lane keeps four
// independent chains in flight (a single chain is latency-bound).
// (x: the pair's values staged in shared memory, or global memory for a pair
// too large to stage)
template <class T>
__device__ __forceinline__ T run8(const T *c, const T *x) {
    T a = c[0] * x[0], b = c[4] * x[4];
#pragma unroll
    for (int e = 1; e < 4; ++e) {
        a = fma(c[e], x[e], a);
        b = fma(c[4 + e], x[4 + e], b);
    }
    return a + b;
}
template <class T>
__device__ __forceinline__ void dot_x1_tail(const T *c, int l, int len, const T *x, KSum<T> &a) {
    for (; l + 8 <= len; l += 8) a.add(run8(c + l, x + l));
    for (; l < len; ++l) a.add(c[l] * x[l]);
}
template <class T>
__device__ __forceinline__ void dot_x1_pair(const T *c0, int len0, const T *x0, const T *c1, int len1, const T *x1,
                                            KSum<T> &a, KSum<T> &b) {
    const int both = min(len0, len1);
    int l = 0;
    for (; l + 8 <= both; l += 8) {
        const T p = run8(c0 + l, x0 + l), q = run8(c1 + l, x1 + l);
        a.add(p);
        b.add(q);
    }
    dot_x1_tail(c0, l, len0, x0, a);
    dot_x1_tail(c1, l, len1, x1, b);
}
// sum over k < r of row[k * ld] t[k] for two rows at once (eight terms per run)
template <class T>
__device__ __forceinline__ T run8_t(const T *row, int ld, const T *t) {
    T a = row[0] * t[0], b = row[4 * ld] * t[4];
#pragma unroll
    for (int e = 1; e < 4; ++e) {
        a = fma(row[e * ld], t[e], a);
        b = fma(row[(4 + e) * ld], t[4 + e], b);
    }
    return a + b;
}
template <class T>
__device__ __forceinline__ void dot_t1_pair(const T *r0, int ld0, const T *t0, const T *r1, int ld1, const T *t1,
                                            int r, bool two, KSum<T> &a, KSum<T> &b) {
    int k = 0;
    for (; k + 8 <= r; k += 8) {
        a.add(run8_t(r0 + k * ld0, ld0, t0 + k));
        if (two) b.add(run8_t(r1 + k * ld1, ld1, t1 + k));
    }
    for (; k < r; ++k) {
        a.add(r0[k * ld0] * t0[k]);
        if (two) b.add(r1[k * ld1] * t1[k]);
    }
}

// FP32, one column, packed pairs of rows (Blackwell's two-lane FP32 FMA): the
// factors' columns start 8-byte aligned (sym_ld), x is staged with each segment
// padded to an even length (zeros), so two terms are one 8-byte load and one
// packed FMA.  run4x2: 8 terms as two 4-term chains (the two halves).
__device__ __forceinline__ float run4x2(const float2 *c, const float2 *x) {
    float2 a = __fmul2_rn(c[0], x[0]);
#pragma unroll
    for (int e = 1; e < 4; ++e) a = __ffma2_rn(c[e], x[e], a);
    return a.x + a.y;
}
__device__ __forceinline__ void dot2_tail(const float2 *c, int p, int np, const float2 *x, KSum<float> &a) {
    for (; p + 4 <= np; p += 4) a.add(run4x2(c + p, x + p));
    for (; p < np; ++p) {
        const float2 q = __fmul2_rn(c[p], x[p]);
        a.add(q.x + q.y);
    }
}
// two dot products at once (np0 and np1 pairs of terms)
__device__ __forceinline__ void dot2_pair(const float2 *c0, int np0, const float2 *x0, const float2 *c1, int np1,
                                          const float2 *x1, KSum<float> &a, KSum<float> &b) {
    const int both = min(np0, np1);
    int p = 0;
    for (; p + 4 <= both; p += 4) {
        const float u = run4x2(c0 + p, x0 + p), v = run4x2(c1 + p, x1 + p);
        a.add(u);
        b.add(v);
    }
    dot2_tail(c0, p, np0, x0, a);
    dot2_tail(c1, p, np1, x1, b);
}
// rows (2p, 2p + 1) of a factor times t: col = &F[2p] (8-byte aligned), column
// stride ld (even); eight k per run in two packed chains, each half of the
// result Kahan-added
__device__ __forceinline__ void rows2_t(const float *col, int ld, int r, const float *t, KSum<float> &a0,
                                        KSum<float> &a1) {
    int k = 0;
    for (; k + 8 <= r; k += 8) {
        float2 u = __fmul2_rn(*reinterpret_cast<const float2 *>(col + (int64_t)k * ld), make_float2(t[k], t[k]));
        float2 v = __fmul2_rn(*reinterpret_cast<const float2 *>(col + (int64_t)(k + 4) * ld),
                              make_float2(t[k + 4], t[k + 4]));
#pragma unroll
        for (int e = 1; e < 4; ++e) {
            u = __ffma2_rn(*reinterpret_cast<const float2 *>(col + (int64_t)(k + e) * ld),
                           make_float2(t[k + e], t[k + e]), u);
            v = __ffma2_rn(*reinterpret_cast<const float2 *>(col + (int64_t)(k + 4 + e) * ld),
                           make_float2(t[k + 4 + e], t[k + 4 + e]), v);
        }
        const float2 w = __fadd2_rn(u, v);
        a0.add(w.x);
        a1.add(w.y);
    }
    for (; k < r; ++k) {
        const float2 w =
            __fmul2_rn(*reinterpret_cast<const float2 *>(col + (int64_t)k * ld), make_float2(t[k], t[k]));
        a0.add(w.x);
        a1.add(w.y);
    }
}
// x_X then x_Y into dst, each padded with zeros to an even length (threads
// tid, tid + nthr, ...)
__device__ __forceinline__ void stage_x2(float *dst, const float *__restrict__ xs, const SymBlk &B, int tid,
                                         int nthr) {
    const int mE = (B.m + 1) & ~1, nE = (B.n + 1) & ~1;
    for (int i = tid; i < mE + nE; i += nthr) {
        float v = 0.f;
        if (i < B.m) v = __ldg(xs + B.xs + i);
        else if (i >= mE && i - mE < B.n) v = __ldg(xs + B.ys + (i - mE));
        dst[i] = v;
    }
}
// the row pairs of U t and V t' (pairs p < PU of U, then of V), threads tid,
// tid + nthr, ...; rows past m (n) are padding and not written
__device__ __forceinline__ void rows2_out(const SymBlk &B, const float *U, const float *V, const float *tt,
                                          const float *tu, double *__restrict__ acc, int tid, int nthr) {
    const int PU = (B.m + 1) >> 1, PV = (B.n + 1) >> 1;
    for (int p = tid; p < PU + PV; p += nthr) {
        const bool xu = p < PU;
        const int r0 = 2 * (xu ? p : p - PU);
        KSum<float> a0, a1;
        rows2_t(xu ? U + r0 : V + r0, xu ? B.ldm : B.ldn, B.r, xu ? tt : tu, a0, a1);
        const int len = xu ? B.m : B.n;
        double *o = acc + (int64_t)(xu ? B.xs : B.ys) + r0;
        atomicAdd(o, (double)a0.get());
        if (r0 + 1 < len) atomicAdd(o + 1, (double)a1.get());
    }
}

// row i of U t (i < m) or of V t' (m <= i < m + n), added to its output row
template <class T, int NQ>
__device__ __forceinline__ void pair_row(const SymBlk &B, const T *U, const T *V, const T *tt, const T *tu, int i,
                                         double *__restrict__ acc) {
    const bool xu = i < B.m;
    const int ii = xu ? i : i - B.m;
    KSum<T> a[NQ];
    dot_t<T, NQ>(xu ? U + ii : V + ii, xu ? B.ldm : B.ldn, B.r, xu ? tt : tu, a);
    const int64_t o = ((int64_t)(xu ? B.xs : B.ys) + ii) * NQ;
#pragma unroll
    for (int q = 0; q < NQ; ++q) atomicAdd(acc + o + q, (double)a[q].get());
}

// One pair by one warp: lane k forms column k of t and t' (the leading
// dimensions keep the lanes' column walks on distinct banks), then lane i
// forms rows i of U t and V t'.  tw: 2 * kSymSmallR * NQ values of this warp.
constexpr int kSymXWarp = 256;   // x values a warp stages for its pair (one column)

template <class T, int NQ>
__device__ __forceinline__ void pair_warp(const SymBlk &B, const T *st, const T *__restrict__ xs,
                                          double *__restrict__ acc, T *tw, T *xw, int lane) {
    const T *U = st, *V = st + (int64_t)B.r * B.ldm;
    T *tt = tw, *tu = tw + kSymSmallR * NQ;
    if constexpr (NQ == 1 && sizeof(T) == 4) {
        const int mE = (B.m + 1) & ~1, nE = (B.n + 1) & ~1;
        if (mE + nE <= kSymXWarp) {   // packed pairs of rows
            stage_x2(xw, xs, B, lane, 32);
            __syncwarp();
            const float2 *xX2 = reinterpret_cast<const float2 *>(xw), *xY2 = reinterpret_cast<const float2 *>(xw + mE);
            for (int k = lane; k < B.r; k += 32) {
                KSum<float> a, c;
                dot2_pair(reinterpret_cast<const float2 *>(V + (int64_t)k * B.ldn), nE >> 1, xY2,
                          reinterpret_cast<const float2 *>(U + (int64_t)k * B.ldm), mE >> 1, xX2, a, c);
                tt[k] = a.get();
                tu[k] = c.get();
            }
            __syncwarp();
            rows2_out(B, U, V, tt, tu, acc, lane, 32);
            __syncwarp();
            return;
        }
    }
    if constexpr (NQ == 1) {
        // x_X and x_Y into the warp's slice with all loads in flight at once (one
        // memory latency per pair instead of one per run of terms)
        const T *xX = xs + B.xs, *xY = xs + B.ys;
        if (B.m + B.n <= kSymXWarp) {
            for (int i = lane; i < B.m; i += 32) xw[i] = __ldg(xs + B.xs + i);
            for (int i = lane; i < B.n; i += 32) xw[B.m + i] = __ldg(xs + B.ys + i);
            __syncwarp();
            xX = xw;
            xY = xw + B.m;
        }
        for (int k = lane; k < B.r; k += 32) {
            KSum<T> a, c;
            dot_x1_pair<T>(V + (int64_t)k * B.ldn, B.n, xY, U + (int64_t)k * B.ldm, B.m, xX, a, c);
            tt[k] = a.get();
            tu[k] = c.get();
        }
        __syncwarp();
        // rows i and i + 32 together: two chains per lane
        const int mn = B.m + B.n;
        for (int i = lane; i < mn; i += 64) {
            const int i2 = i + 32;
            const bool two = i2 < mn;
            const bool u0 = i < B.m, u1 = i2 < B.m;
            const int a0 = u0 ? i : i - B.m, a1 = u1 ? i2 : i2 - B.m;
            KSum<T> a, b;
            dot_t1_pair<T>(u0 ? U + a0 : V + a0, u0 ? B.ldm : B.ldn, u0 ? tt : tu, u1 ? U + a1 : V + a1,
                           u1 ? B.ldm : B.ldn, u1 ? tt : tu, B.r, two, a, b);
            atomicAdd(acc + (int64_t)(u0 ? B.xs : B.ys) + a0, (double)a.get());
            if (two) atomicAdd(acc + (int64_t)(u1 ? B.xs : B.ys) + a1, (double)b.get());
        }
    } else {
        for (int k = lane; k < B.r; k += 32) {
            KSum<T> a[NQ], c[NQ];
            dot_x<T, NQ>(V + (int64_t)k * B.ldn, B.n, xs, B.ys, a);
            dot_x<T, NQ>(U + (int64_t)k * B.ldm, B.m, xs, B.xs, c);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                tt[k * NQ + q] = a[q].get();
                tu[k * NQ + q] = c[q].get();
            }
        }
        __syncwarp();
        for (int i = lane; i < B.m + B.n; i += 32) pair_row<T, NQ>(B, U, V, tt, tu, i, acc);
    }
    __syncwarp();
}

// One pair by the whole CTA: warp w forms the columns w, w + NW, ... of t and t'
// (lanes over the rows, then a butterfly sum), then thread i rows i of U t and
// V t'.  tb: 2 * kSymMaxR * NQ values.
template <class T, int NQ, int NW>
__device__ __forceinline__ void pair_cta(const SymBlk &B, const T *st, const T *__restrict__ xs,
                                         double *__restrict__ acc, T *tb, T *xb, int warp, int lane) {
    const T *U = st, *V = st + (int64_t)B.r * B.ldm;
    T *tt = tb, *tu = tb + kSymMaxR * NQ;
    if constexpr (NQ == 1 && sizeof(T) == 4) {
        const int mE = (B.m + 1) & ~1, nE = (B.n + 1) & ~1;
        if (mE + nE <= NW * kSymXWarp) {   // packed pairs of rows
            stage_x2(xb, xs, B, threadIdx.x, NW * 32);
            __syncthreads();
            const float2 *xX2 = reinterpret_cast<const float2 *>(xb), *xY2 = reinterpret_cast<const float2 *>(xb + mE);
            // column k of V and of U: lanes over pairs of rows, then a butterfly sum
            for (int k = warp; k < B.r; k += NW) {
                KSum<float> a, c;
                const float2 *cv = reinterpret_cast<const float2 *>(V + (int64_t)k * B.ldn);
                const float2 *cu = reinterpret_cast<const float2 *>(U + (int64_t)k * B.ldm);
                const int mx = max(mE, nE) >> 1;
                for (int q = lane; q < mx; q += 32) {
                    if (2 * q < nE) {
                        const float2 w = __fmul2_rn(cv[q], xY2[q]);
                        a.add(w.x + w.y);
                    }
                    if (2 * q < mE) {
                        const float2 w = __fmul2_rn(cu[q], xX2[q]);
                        c.add(w.x + w.y);
                    }
                }
                float v = a.get(), w = c.get();
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    v += __shfl_xor_sync(0xffffffffu, v, o);
                    w += __shfl_xor_sync(0xffffffffu, w, o);
                }
                if (lane == 0) {
                    tt[k] = v;
                    tu[k] = w;
                }
            }
            __syncthreads();
            rows2_out(B, U, V, tt, tu, acc, threadIdx.x, NW * 32);
            return;
        }
    }
    if constexpr (NQ == 1) {
        const T *xX = xs + B.xs, *xY = xs + B.ys;
        if (B.m + B.n <= NW * kSymXWarp) {   // x_X and x_Y staged by the whole CTA
            for (int i = threadIdx.x; i < B.m + B.n; i += NW * 32)
                xb[i] = i < B.m ? __ldg(xs + B.xs + i) : __ldg(xs + B.ys + (i - B.m));
            __syncthreads();
            xX = xb;
            xY = xb + B.m;
        }
        // column k of V and of U together (two chains per lane)
        for (int k = warp; k < B.r; k += NW) {
            KSum<T> a, c;
            const T *cv = V + (int64_t)k * B.ldn, *cu = U + (int64_t)k * B.ldm;
            const int mx = max(B.m, B.n);
            for (int j = lane; j < mx; j += 32) {
                if (j < B.n) a.add(cv[j] * xY[j]);
                if (j < B.m) c.add(cu[j] * xX[j]);
            }
            T v = a.get(), w = c.get();
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                v += __shfl_xor_sync(0xffffffffu, v, o);
                w += __shfl_xor_sync(0xffffffffu, w, o);
            }
            if (lane == 0) {
                tt[k] = v;
                tu[k] = w;
            }
        }
        __syncthreads();
        const int mn = B.m + B.n;
        for (int i = threadIdx.x; i < mn; i += 2 * NW * 32) {
            const int i2 = i + NW * 32;
            const bool two = i2 < mn;
            const bool u0 = i < B.m, u1 = i2 < B.m;
            const int a0 = u0 ? i : i - B.m, a1 = u1 ? i2 : i2 - B.m;
            KSum<T> a, b;
            dot_t1_pair<T>(u0 ? U + a0 : V + a0, u0 ? B.ldm : B.ldn, u0 ? tt : tu, u1 ? U + a1 : V + a1,
                           u1 ? B.ldm : B.ldn, u1 ? tt : tu, B.r, two, a, b);
            atomicAdd(acc + (int64_t)(u0 ? B.xs : B.ys) + a0, (double)a.get());
            if (two) atomicAdd(acc + (int64_t)(u1 ? B.xs : B.ys) + a1, (double)b.get());
        }
        return;
    }
    for (int d = warp; d < 2 * B.r; d += NW) {
        const bool isv = d < B.r;
        const int k = isv ? d : d - B.r;
        const T *col = isv ? V + (int64_t)k * B.ldn : U + (int64_t)k * B.ldm;
        const int len = isv ? B.n : B.m;
        const int64_t x0 = isv ? B.ys : B.xs;
        KSum<T> a[NQ];
        for (int j = lane; j < len; j += 32) {
            T x[NQ];
            load_x<T, NQ>(xs, x0 + j, x);
            const T cj = col[j];
#pragma unroll
            for (int q = 0; q < NQ; ++q) a[q].add(cj * x[q]);
        }
        T v[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            v[q] = a[q].get();
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        }
        if (lane == 0) {
            T *dst = isv ? tt : tu;
#pragma unroll
            for (int q = 0; q < NQ; ++q) dst[k * NQ + q] = v[q];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < B.m + B.n; i += NW * 32) pair_row<T, NQ>(B, U, V, tt, tu, i, acc);
}

constexpr int kSymWarps1 = 16, kSymWarps8 = 8;   // warps per CTA for 1 and 8 columns

template <class T, int NQ, int NW>
__host__ __device__ constexpr size_t tbuf_elems() {
    return (size_t)(NW * kSymSmallR * NQ * 2 > kSymMaxR * NQ * 2 ? NW * kSymSmallR * NQ * 2 : kSymMaxR * NQ * 2);
}

template <class T, int NQ, int NW>
__host__ __device__ constexpr size_t xbuf_elems() {
    return NQ == 1 ? (size_t)NW * kSymXWarp : 0;
}

template <class T, int NQ, int NW>
constexpr size_t sym_smem() {
    return 2 * (size_t)(sizeof(T) == 8 ? kSymStageF64 : kSymStageF32) +
           (tbuf_elems<T, NQ, NW>() + xbuf_elems<T, NQ, NW>()) * sizeof(T);
}

// Persistent: CTA c takes groups c, c + gridDim.x, ...; group j of a CTA lands
// in stage j % 2, the copy of group j + 2 is issued once group j is done.
// (one column: at most 80 registers, so that the other pairs' gather and the
// near field have room on every SM beside it)
template <class T, int NQ, int NW>
__global__ void __maxnreg__(NQ == 1 ? 80 : 65536 / (NW * 32)) k_sym(SymArgs S, const T *__restrict__ xs,
                                                                   double *__restrict__ acc) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[2];
    T *tbuf = reinterpret_cast<T *>(smem + 2 * (size_t)S.stage);
    T *xbuf = tbuf + tbuf_elems<T, NQ, NW>();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g0 = blockIdx.x, gs = gridDim.x;
    const int nmine = g0 < S.ngrp ? (S.ngrp - g0 + gs - 1) / gs : 0;
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const uint64_t pol = l2_evict_first_policy();   // the factors are read once: keep x and acc in L2
    auto issue = [&](int j) {
        const SymGroup G = S.grp[g0 + j * gs];
        mbar_arrive_expect_tx(&bars[j & 1], (uint32_t)G.bytes);
        bulk_copy_g2s_hint(smem + (size_t)(j & 1) * S.stage, S.F + G.off * (int64_t)sizeof(T), (uint32_t)G.bytes,
                           &bars[j & 1], pol);
    };
    if (threadIdx.x == 0)
        for (int j = 0; j < min(2, nmine); ++j) issue(j);
    for (int j = 0; j < nmine; ++j) {
        const bool ok = mbar_wait(&bars[j & 1], (uint32_t)(j >> 1) & 1u);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                *S.err = H3D_ERR_TIMEOUT;
                for (int q = j; q < min(j + 2, nmine); ++q) mbar_wait(&bars[q & 1], (uint32_t)(q >> 1) & 1u);
            }
            return;
        }
        const SymGroup G = S.grp[g0 + j * gs];
        const T *st = reinterpret_cast<const T *>(smem + (size_t)(j & 1) * S.stage);
        if (G.big) {
            pair_cta<T, NQ, NW>(S.blk[G.b0], st, xs, acc, tbuf, xbuf, warp, lane);
        } else {
            T *tw = tbuf + (size_t)warp * kSymSmallR * NQ * 2;
            T *xw = xbuf + (size_t)warp * kSymXWarp;
            for (int p = warp; p < G.nb; p += NW) {
                const SymBlk B = S.blk[G.b0 + p];
                pair_warp<T, NQ>(B, st + (B.off - G.off), xs, acc, tw, xw, lane);
            }
        }
        __syncthreads();   // stage j % 2 and the coefficient buffer are free again
        if (threadIdx.x == 0 && j + 2 < nmine) issue(j + 2);
    }
}

template <class T>
__global__ void k_sym_add(T *__restrict__ out, const double *__restrict__ acc, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = (T)((double)out[e] + acc[e]);
}

template <class T, int NQ, int NW>
void launch_sym(Handle &h, const T *xs, cudaStream_t s) {
    SymArgs A{h.sym_blk, h.sym_grp, h.nsym_grp, sizeof(T) == 8 ? kSymStageF64 : kSymStageF32,
              static_cast<const unsigned char *>(h.symF), h.d_async_err};
    const int grid = std::min(h.nsym_grp, num_sms());
    k_sym<T, NQ, NW><<<grid, NW * 32, sym_smem<T, NQ, NW>(), s>>>(A, xs, h.sym_acc);
    H3D_LAUNCH_CHECK();
}

}  // namespace

void sym_prepare() {
    static bool done = false;
    if (done) return;
    H3D_CUDA(cudaFuncSetAttribute(k_sym<float, 1, kSymWarps1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sym_smem<float, 1, kSymWarps1>()));
    H3D_CUDA(cudaFuncSetAttribute(k_sym<float, 8, kSymWarps8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sym_smem<float, 8, kSymWarps8>()));
    H3D_CUDA(cudaFuncSetAttribute(k_sym<double, 1, kSymWarps1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sym_smem<double, 1, kSymWarps1>()));
    H3D_CUDA(cudaFuncSetAttribute(k_sym<double, 8, kSymWarps8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sym_smem<double, 8, kSymWarps8>()));
    done = true;
}

void sym_product(Handle &h, const void *xs, int nq, cudaStream_t s, cudaEvent_t ev) {
    if (h.nsym_grp == 0) return;
    cudaStream_t ss = h.sym_stream;
    H3D_CUDA(cudaEventRecord(h.ev_sym_fork, s));
    H3D_CUDA(cudaStreamWaitEvent(ss, h.ev_sym_fork, 0));
    H3D_CUDA(cudaMemsetAsync(h.sym_acc, 0, (size_t)h.N * nq * sizeof(double), ss));
    if (h.prec == H3D_FP64) {
        if (nq == 1) launch_sym<double, 1, kSymWarps1>(h, (const double *)xs, ss);
        else launch_sym<double, 8, kSymWarps8>(h, (const double *)xs, ss);
    } else {
        if (nq == 1) launch_sym<float, 1, kSymWarps1>(h, (const float *)xs, ss);
        else launch_sym<float, 8, kSymWarps8>(h, (const float *)xs, ss);
    }
    if (ev) H3D_CUDA(cudaEventRecord(ev, ss));
    H3D_CUDA(cudaEventRecord(h.ev_sym_join, ss));
}

void sym_finish(Handle &h, void *out, int nq, cudaStream_t s) {
    if (h.nsym_grp == 0) return;
    H3D_CUDA(cudaStreamWaitEvent(s, h.ev_sym_join, 0));
    const int64_t n = h.N * nq;
    const unsigned grid = (unsigned)std::max<int64_t>(1, (n + 255) / 256);
    if (h.prec == H3D_FP64) k_sym_add<double><<<grid, 256, 0, s>>>((double *)out, h.sym_acc, n);
    else k_sym_add<float><<<grid, 256, 0, s>>>((float *)out, h.sym_acc, n);
    H3D_LAUNCH_CHECK();
}

}  // namespace h3d
