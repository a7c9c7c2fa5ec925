// h3d_forces.cu -- forces F = -dE/dp on the points for the energy
//   E = 1/2 q^T A~ q
// of the HODLR3D operator with its ACA pivots frozen.  The near blocks are exact
// kernel entries; every admissible block (X, Y) with row pivots sigma and column
// pivots tau is the cross form of the paper's ACA (Sec. 4.1, Eq. prank),
//   A_XY = K(X,tau) M^{-1} K(sigma,Y),   M = K(sigma,tau).
// With s = K(sigma,Y) q_Y, c = M^{-1} s, u = K(X,tau)^T q_X and a = M^{-T} u the
// block's energy 1/2 u^T c has the differential
//   1/2 [ q_X^T dK(X,tau) c + a^T dK(sigma,Y) q_Y - a^T dM c ],
// and each kernel entry K(p_i, p_j) = f(|p_i - p_j|) differentiates to
// g = f'(rho) (p_i - p_j) / rho for p_i and -g for p_j.  Kernel entries are
// recomputed (nothing is stored).  The admissible blocks are evaluated in FP64
// for every handle: c and a carry the condition of M (up to ~1e7), and the
// terms at the pivot points cancel to the interpolation error, so an FP32 entry
// error of 1e-7 would be amplified past the result.  M is factored by Gaussian
// elimination with partial pivoting.  The near field of FP32 handles evaluates
// in FP32 (coordinate differences from a hi + lo split, compensated sums).
// Far-field contributions reach the points through FP64 atomic additions; the
// energy is reduced in a fixed order.
#include "h3d_ff.cuh"
#include "h3d_internal.cuh"

namespace h3d {
namespace {

constexpr int kFThreads = 128;
constexpr int kFWarps = kFThreads / 32;

// 1/sqrt(d2) to FP64 accuracy without the FP64 square root or division: an
// FP32 seed y0 = y (1 + delta), |delta| < 2^-21, then one third-order step of
// the binomial series y = y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3 e^2/8 + ...) with
// e = 1 - d2 y0^2 (y0^2 is exact in FP64: y0 has 24 significant bits); the
// neglected terms are below 5/16 |e|^3 < 2^-60.  Five FP64 operations.
__device__ __forceinline__ double rsqrt64(double d2) {
    const double y0 = (double)rsqrtf((float)d2);
    const double e = fma(-d2, y0 * y0, 1.0);
    return fma(y0 * e, fma(0.375, e, 0.5), y0);
}

// K(rho) and f'(rho) / rho from rho^2 (both 0 at rho = 0): the gradient of
// K(|a - b|) with respect to a is fr (a - b).
__device__ __forceinline__ double kval_fr(int kind, double kappa, double d2, double &fr) {
    if (d2 == 0.0) {
        fr = 0.0;
        return 0.0;
    }
    const double ir = rsqrt64(d2), ir2 = ir * ir;
    double f;
    switch (kind) {
    case H3D_LAPLACE: f = H3D_INV4PI * ir; fr = -f * ir2; break;
    case H3D_YUKAWA: {
        const double r = d2 * ir;
        f = H3D_INV4PI * exp(-kappa * r) * ir;
        fr = -f * (1.0 + kappa * r) * ir2;
        break;
    }
    case H3D_INV_R4: f = ir2 * ir2; fr = -4.0 * f * ir2; break;
    default: {
        const double r = d2 * ir;
        double sn, cs;
        sincos(r, &sn, &cs);
        f = cs * ir;
        fr = -(r * sn + cs) * ir2 * ir;
    }
    }
    return f;
}

// K(a, b) and dK/da = (f'(rho) / rho) (a - b) for a - b = (dx, dy, dz)
__device__ __forceinline__ double kval_grad(int kind, double kappa, double dx, double dy, double dz, double &gx,
                                            double &gy, double &gz) {
    double fr;
    const double f = kval_fr(kind, kappa, dx * dx + dy * dy + dz * dz, fr);
    gx = fr * dx;
    gy = fr * dy;
    gz = fr * dz;
    return f;
}

__device__ __forceinline__ float kval_grad(int kind, float kappa, float dx, float dy, float dz, float &gx, float &gy,
                                           float &gz) {
    const float d2 = dx * dx + dy * dy + dz * dz;
    if (d2 == 0.0f) {
        gx = gy = gz = 0.0f;
        return 0.0f;
    }
    const float ir = rsqrtf(d2), r = d2 * ir;
    float f, fr;
    switch (kind) {
    case H3D_LAPLACE: f = (float)H3D_INV4PI * ir; fr = -f * ir * ir; break;
    case H3D_YUKAWA: f = (float)H3D_INV4PI * expf(-kappa * r) * ir; fr = -f * (1.0f + kappa * r) * ir * ir; break;
    case H3D_INV_R4: f = (ir * ir) * (ir * ir); fr = -4.0f * f * ir * ir; break;
    default: {
        float sn, cs;
        sincosf(r, &sn, &cs);
        f = cs * ir;
        fr = -(r * sn + cs) * ir * ir * ir;
    }
    }
    gx = fr * dx;
    gy = fr * dy;
    gz = fr * dz;
    return f;
}

// sums of evaluations: plain in FP64, compensated (Kahan) in FP32
template <class T> struct KSum;
template <> struct KSum<double> {
    double s = 0.0;
    __device__ void add(double v) { s += v; }
    __device__ double get() const { return s; }
};
template <> struct KSum<float> {
    float s = 0.f, c = 0.f;
    __device__ void add(float v) {
        const float y = v - c, t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ double get() const { return (double)s - (double)c; }
};

struct ForceArgs {
    int kind;
    double kappa;
    const double *px, *py, *pz;
    const float4 *ph, *pl;     // FP32 evaluation: coordinates split hi + lo, charge in ph.w
    const double *qs;          // charges, Morton order
    double *G;                 // dE/dp, Morton order, N x 3
    // near
    int64_t offL;
    int nleaf;
    const int *box_start, *box_end, *near_ptr, *near_src;
    // far
    int64_t nblk;
    const int *blk_tgt, *blk_src, *rank, *sigma, *tau;
    const int64_t *piv_off;
    double *Mscr;              // mr^2 per CTA
    int mr;                    // largest rank of the handle
    double *Epart;             // per leaf (near), then per block (far)
    int *next;                 // far-field work queue head (zero before the launch)
};

// p_i - p_j in the evaluation type: FP64 directly; FP32 from the hi + lo split
// (each FP32 subtraction is correctly rounded, so the difference keeps ~1e-7 of
// its own size, not of the coordinates)
__device__ __forceinline__ void pdiff(const ForceArgs &A, int i, int j, double &dx, double &dy, double &dz) {
    dx = A.px[i] - A.px[j];
    dy = A.py[i] - A.py[j];
    dz = A.pz[i] - A.pz[j];
}
__device__ __forceinline__ void pdiff(const ForceArgs &A, int i, int j, float &dx, float &dy, float &dz) {
    const float4 hi = A.ph[i], hj = A.ph[j], li = A.pl[i], lj = A.pl[j];
    dx = (hi.x - hj.x) + (li.x - lj.x);
    dy = (hi.y - hj.y) + (li.y - lj.y);
    dz = (hi.z - hj.z) + (li.z - lj.z);
}
template <class T> __device__ __forceinline__ T charge(const ForceArgs &A, int i);
template <> __device__ __forceinline__ double charge<double>(const ForceArgs &A, int i) { return A.qs[i]; }
template <> __device__ __forceinline__ float charge<float>(const ForceArgs &A, int i) { return A.ph[i].w; }

template <class T>
__global__ void k_charges_sorted(const T *__restrict__ q, const int *__restrict__ perm, const double *__restrict__ px,
                                 const double *__restrict__ py, const double *__restrict__ pz, int64_t n,
                                 double *__restrict__ qs, float4 *__restrict__ ph, float4 *__restrict__ pl) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double q64 = (double)q[perm[s]];
    qs[s] = q64;
    if (ph) {
        const float xh = (float)px[s], yh = (float)py[s], zh = (float)pz[s];
        ph[s] = make_float4(xh, yh, zh, (float)q64);
        pl[s] = make_float4((float)(px[s] - xh), (float)(py[s] - yh), (float)(pz[s] - zh), 0.f);
    }
}

__device__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kFWarps; ++w) t += red[w];
    __syncthreads();
    return t;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// near field: every point of a leaf against every point of its near leaves
template <class T>
__global__ void __launch_bounds__(kFThreads) k_force_near(ForceArgs A) {
    __shared__ double red[kFWarps];
    const int z = blockIdx.x;
    const int Zg = (int)(A.offL + z);
    const int x0 = A.box_start[Zg], x1 = A.box_end[Zg];
    double e = 0.0;
    for (int i = x0 + threadIdx.x; i < x1; i += kFThreads) {
        KSum<T> ei, gx, gy, gz;
        for (int p = A.near_ptr[z]; p < A.near_ptr[z + 1]; ++p) {
            const int Sg = (int)(A.offL + A.near_src[p]);
            for (int j = A.box_start[Sg]; j < A.box_end[Sg]; ++j) {
                if (j == i) continue;
                T dx, dy, dz, hx, hy, hz;
                pdiff(A, i, j, dx, dy, dz);
                const T k = kval_grad(A.kind, (T)A.kappa, dx, dy, dz, hx, hy, hz);
                const T qj = charge<T>(A, j);
                ei.add(qj * k);
                gx.add(qj * hx);
                gy.add(qj * hy);
                gz.add(qj * hz);
            }
        }
        const double qi = A.qs[i];
        e += 0.5 * qi * ei.get();
        A.G[3 * (int64_t)i] = qi * gx.get();
        A.G[3 * (int64_t)i + 1] = qi * gy.get();
        A.G[3 * (int64_t)i + 2] = qi * gz.get();
    }
    const double t = block_sum(e, red);
    if (threadIdx.x == 0) A.Epart[z] = t;
}

__device__ __forceinline__ void gadd(double *G, int p, double s, double gx, double gy, double gz) {
    atomicAdd(G + 3 * (int64_t)p, s * gx);
    atomicAdd(G + 3 * (int64_t)p + 1, s * gy);
    atomicAdd(G + 3 * (int64_t)p + 2, s * gz);
}

// P M = L U with partial pivoting (ties: the smaller row) by one warp for r <= 32,
// lane i owning row i of M (row-major in the CTA's scratch), then
//   c = U^{-1} L^{-1} P s   (s given in c),  the block energy 1/2 u^T c,
//   a = P^T L^{-T} U^{-T} u (u given in a and u0);  piv[k] = original row of row k.
// The same operations as the CTA-wide path, in one warp and without barriers.
__device__ void factor_solve_warp(double *M, int r, double *c, double *a, const double *u0, int *piv, double *Eout,
                                  int lane) {
    const int i = lane;
    const bool row = i < r;
    double ci = row ? c[i] : 0.0;
    int pi = i;
    for (int k = 0; k < r; ++k) {
        double v = (row && i >= k) ? fabs(M[(size_t)i * r + k]) : -1.0;
        int bi = i;
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, v, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > v || (ov == v && oi < bi)) { v = ov; bi = oi; }
        }
        // lane 0's choice for every lane (uniform even if a value were not finite),
        // and every shuffle outside the branch
        const int p = __shfl_sync(0xffffffffu, bi, 0);
        const double cvk = __shfl_sync(0xffffffffu, ci, k), cvp = __shfl_sync(0xffffffffu, ci, p);
        const int pk = __shfl_sync(0xffffffffu, pi, k), pp = __shfl_sync(0xffffffffu, pi, p);
        if (p != k) {
            for (int j = lane; j < r; j += 32) {
                const double t = M[(size_t)k * r + j];
                M[(size_t)k * r + j] = M[(size_t)p * r + j];
                M[(size_t)p * r + j] = t;
            }
            if (i == k) { ci = cvp; pi = pp; }
            if (i == p) { ci = cvk; pi = pk; }
        }
        __syncwarp();
        const double ck = __shfl_sync(0xffffffffu, ci, k);
        if (row && i > k) {
            const double l = M[(size_t)i * r + k] / M[(size_t)k * r + k];
            M[(size_t)i * r + k] = l;
            for (int j = k + 1; j < r; ++j) M[(size_t)i * r + j] = fma(-l, M[(size_t)k * r + j], M[(size_t)i * r + j]);
            ci = fma(-l, ck, ci);
        }
        __syncwarp();
    }
    for (int k = r - 1; k >= 0; --k) {   // U c = z
        if (i == k) ci = ci / M[(size_t)k * r + k];
        const double ck = __shfl_sync(0xffffffffu, ci, k);
        if (row && i < k) ci = fma(-M[(size_t)i * r + k], ck, ci);
    }
    double e = row ? 0.5 * u0[i] * ci : 0.0;
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0) *Eout = e;
    double ai = row ? a[i] : 0.0;
    for (int k = 0; k < r; ++k) {   // U^T z = u
        if (i == k) ai = ai / M[(size_t)k * r + k];
        const double ak = __shfl_sync(0xffffffffu, ai, k);
        if (row && i > k) ai = fma(-M[(size_t)k * r + i], ak, ai);
    }
    for (int k = r - 1; k >= 0; --k) {   // L^T w = z (unit diagonal)
        const double wk = __shfl_sync(0xffffffffu, ai, k);
        if (row && i < k) ai = fma(-M[(size_t)k * r + i], wk, ai);
    }
    __syncwarp();
    if (row) {
        c[i] = ci;
        piv[i] = pi;
        a[pi] = ai;   // a <- P^T w
    }
}

// far field: one block at a time per CTA (taken from a queue), M in this CTA's
// scratch.  FF_ = false: everything in FP64.  FF_ = true (FP32 handles of the
// Laplace and 1/r^4 kernels): the entries of K(sigma,Y), K(X,tau) and their
// gradients, and the sums over the points, in float-float on the FP32 pipes
// (coordinates split hi + lo, FP32 charges exact); M, its factorisation, the
// solves and the -a^T dM c term stay FP64.
// per-block arrays in dynamic shared memory, sized by the largest rank mr:
// c, a, u0 (mr doubles each), gs, gt (3 mr doubles each), sp, tp, piv (mr ints)
inline size_t far_smem(int mr) { return (size_t)mr * (9 * sizeof(double) + 3 * sizeof(int)); }
constexpr int kFarCtasMax = 7;   // per SM (72 registers; fewer when mr makes the arrays large)

template <bool FF_>
__global__ void __launch_bounds__(kFThreads, kFarCtasMax) k_force_far(ForceArgs A) {
    using T = double;
    extern __shared__ __align__(16) unsigned char fsm[];
    double *c = reinterpret_cast<double *>(fsm), *a = c + A.mr, *u0 = a + A.mr;
    double(*gs)[3] = reinterpret_cast<double(*)[3]>(u0 + A.mr);   // sum_j q_j dK(sigma_k, p_j)
    double(*gt)[3] = gs + A.mr;                                     // sum_i q_i dK(p_i, tau_k)
    int *sp = reinterpret_cast<int *>(gt + A.mr), *tp = sp + A.mr, *piv = tp + A.mr;
    __shared__ double red[kFWarps];
    __shared__ int pmax, sblk[2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    double *M = A.Mscr + (size_t)blockIdx.x * A.mr * A.mr;
    for (int it = 0;; ++it) {
        // blocks in list order (largest first) from a queue: a CTA takes the next
        // block when it is done, so uneven blocks balance over the CTAs
        if (tid == 0) sblk[it & 1] = atomicAdd(A.next, 1);
        __syncthreads();
        const int64_t b = sblk[it & 1];
        if (b >= A.nblk) break;
        const int r = A.rank[b];
        if (r == 0) {
            if (tid == 0) A.Epart[A.nleaf + b] = 0.0;
            continue;
        }
        const int X = A.blk_tgt[b], Y = A.blk_src[b];
        const int x0 = A.box_start[X], m = A.box_end[X] - x0;
        const int y0 = A.box_start[Y], n = A.box_end[Y] - y0;
        const int *sg = A.sigma + A.piv_off[b], *ta = A.tau + A.piv_off[b];
        for (int k = tid; k < r; k += kFThreads) {
            sp[k] = x0 + sg[k];
            tp[k] = y0 + ta[k];
        }
        __syncthreads();
        // one warp per pivot, each entry evaluated once for its value and gradient:
        //   s = K(sigma, Y) q_Y -> c,  u = K(X, tau)^T q_X -> a, u0,
        //   gs_k = sum_j q_j dK(sigma_k, p_j),  gt_k = sum_i q_i dK(p_i, tau_k)
        for (int k = warp; k < r && FF_; k += kFWarps) {
            const int ps = sp[k], pt = tp[k];
            const float4 hs = A.ph[ps], ls = A.pl[ps], ht = A.ph[pt], lt = A.pl[pt];
            FF sv{0.f, 0.f}, uv{0.f, 0.f}, sg[3], tg[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) sg[a] = tg[a] = FF{0.f, 0.f};
            for (int o = lane; o < max(m, n); o += 32) {
                if (o < n) {
                    const float4 hj = A.ph[y0 + o], lj = A.pl[y0 + o];
                    FF f, fr, d[3];
                    ff_kernel_grad(A.kind, hs, ls, hj, lj, f, fr, d);
                    sv = ff_fma_acc(sv, f, hj.w);
                    FF w = ff_two_prod(fr.h, hj.w);
                    w.l = __fmaf_rn(fr.l, hj.w, w.l);
#pragma unroll
                    for (int a = 0; a < 3; ++a) sg[a] = ff_fma_acc(sg[a], w, d[a]);
                }
                if (o < m) {
                    const float4 hi = A.ph[x0 + o], li = A.pl[x0 + o];
                    FF f, fr, d[3];
                    ff_kernel_grad(A.kind, hi, li, ht, lt, f, fr, d);
                    uv = ff_fma_acc(uv, f, hi.w);
                    FF w = ff_two_prod(fr.h, hi.w);
                    w.l = __fmaf_rn(fr.l, hi.w, w.l);
#pragma unroll
                    for (int a = 0; a < 3; ++a) tg[a] = ff_fma_acc(tg[a], w, d[a]);
                }
            }
            sv = ff_warp_sum(sv);
            uv = ff_warp_sum(uv);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                sg[a] = ff_warp_sum(sg[a]);
                tg[a] = ff_warp_sum(tg[a]);
            }
            if (lane == 0) {
                c[k] = ff_to_double(sv);
                a[k] = u0[k] = ff_to_double(uv);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    gs[k][q] = ff_to_double(sg[q]);
                    gt[k][q] = ff_to_double(tg[q]);
                }
            }
        }
        for (int k = warp; k < r && !FF_; k += kFWarps) {
            const int ps = sp[k], pt = tp[k];
            double sv = 0.0, uv = 0.0, s0 = 0.0, s1 = 0.0, s2 = 0.0, t0 = 0.0, t1 = 0.0, t2 = 0.0;
            // the row of sigma_k and the column of tau_k side by side: two independent
            // evaluation chains per lane (the FP64 pipe's latency is long)
            for (int o = lane; o < max(m, n); o += 32) {
                if (o < n) {
                    const int j = y0 + o;
                    double dx, dy, dz, fr;
                    pdiff(A, ps, j, dx, dy, dz);
                    const double qj = A.qs[j];
                    const double f = kval_fr(A.kind, A.kappa, fma(dz, dz, fma(dy, dy, dx * dx)), fr);
                    const double w = qj * fr;
                    sv = fma(f, qj, sv);
                    s0 = fma(w, dx, s0);
                    s1 = fma(w, dy, s1);
                    s2 = fma(w, dz, s2);
                }
                if (o < m) {
                    const int i = x0 + o;
                    double dx, dy, dz, fr;
                    pdiff(A, i, pt, dx, dy, dz);
                    const double qi = A.qs[i];
                    const double f = kval_fr(A.kind, A.kappa, fma(dz, dz, fma(dy, dy, dx * dx)), fr);
                    const double w = qi * fr;
                    uv = fma(qi, f, uv);
                    t0 = fma(w, dx, t0);
                    t1 = fma(w, dy, t1);
                    t2 = fma(w, dz, t2);
                }
            }
            sv = warp_sum(sv); uv = warp_sum(uv);
            s0 = warp_sum(s0); s1 = warp_sum(s1); s2 = warp_sum(s2);
            t0 = warp_sum(t0); t1 = warp_sum(t1); t2 = warp_sum(t2);
            if (lane == 0) {
                c[k] = sv;
                a[k] = uv;
                u0[k] = uv;
                gs[k][0] = s0; gs[k][1] = s1; gs[k][2] = s2;
                gt[k][0] = t0; gt[k][1] = t1; gt[k][2] = t2;
            }
        }
        // M = K(sigma, tau), row-major r x r, FP64 (two entries per thread and step;
        // FF_: float-float entries rounded to FP64)
        for (int e = tid; e < r * r && FF_; e += kFThreads) {
            const int k = e / r, l = e - k * r;
            M[e] = ff_to_double(ff_kernel(A.kind, A.ph[sp[k]], A.pl[sp[k]], A.ph[tp[l]], A.pl[tp[l]]));
        }
        for (int e = tid; e < r * r && !FF_; e += 2 * kFThreads) {
            const int e2 = e + kFThreads;
            const int k = e / r, l = e - k * r;
            double dx, dy, dz, fr;
            pdiff(A, sp[k], tp[l], dx, dy, dz);
            const double v = kval_fr(A.kind, A.kappa, fma(dz, dz, fma(dy, dy, dx * dx)), fr);
            if (e2 < r * r) {
                const int k2 = e2 / r, l2 = e2 - k2 * r;
                pdiff(A, sp[k2], tp[l2], dx, dy, dz);
                M[e2] = kval_fr(A.kind, A.kappa, fma(dz, dz, fma(dy, dy, dx * dx)), fr);
            }
            M[e] = v;
        }
        __syncthreads();   // M, s (in c) and u (in a, u0) are complete
        if (r <= 32) {   // one warp factors and solves, lane i owning row i: no CTA barriers
            if (warp == 0) factor_solve_warp(M, r, c, a, u0, piv, A.Epart + A.nleaf + b, lane);
            __syncthreads();
        } else {
            for (int k = tid; k < r; k += kFThreads) piv[k] = k;
            __syncthreads();
            // energy of the block: 1/2 u^T c with c = M^{-1} s (after the solves)
            // P M = L U (partial pivoting), the row swaps applied to c as well
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
                    for (int j = tid; j < r; j += kFThreads) {
                        const double t = M[(size_t)k * r + j];
                        M[(size_t)k * r + j] = M[(size_t)p * r + j];
                        M[(size_t)p * r + j] = t;
                    }
                    if (tid == 0) {
                        const double t = c[k]; c[k] = c[p]; c[p] = t;
                        const int ti = piv[k]; piv[k] = piv[p]; piv[p] = ti;
                    }
                }
                __syncthreads();
                const double d = M[(size_t)k * r + k];
                for (int i = k + 1 + tid; i < r; i += kFThreads) M[(size_t)i * r + k] /= d;   // L multipliers
                __syncthreads();
                const int rem = r - k - 1;
                for (int e = tid; e < rem * rem; e += kFThreads) {
                    const int i = k + 1 + e / rem, j = k + 1 + e % rem;
                    M[(size_t)i * r + j] -= M[(size_t)i * r + k] * M[(size_t)k * r + j];
                }
                if (tid == 0)
                    for (int i = k + 1; i < r; ++i) c[i] -= M[(size_t)i * r + k] * c[k];
                __syncthreads();
            }
            // c = U^{-1} (L^{-1} P s);  a = P^T L^{-T} U^{-T} u
            for (int k = r - 1; k >= 0; --k) {
                double t = 0.0;
                for (int j = k + 1 + tid; j < r; j += kFThreads) t += M[(size_t)k * r + j] * c[j];
                t = block_sum(t, red);
                if (tid == 0) c[k] = (c[k] - t) / M[(size_t)k * r + k];
                __syncthreads();
            }
            {   // energy 1/2 u^T c, u still intact in u0
                double e = 0.0;
                for (int k = tid; k < r; k += kFThreads) e += 0.5 * u0[k] * c[k];
                e = block_sum(e, red);
                if (tid == 0) A.Epart[A.nleaf + b] = e;
            }
            for (int k = 0; k < r; ++k) {   // U^T z = u (z in a)
                double t = 0.0;
                for (int l = tid; l < k; l += kFThreads) t += M[(size_t)l * r + k] * a[l];
                t = block_sum(t, red);
                if (tid == 0) a[k] = (a[k] - t) / M[(size_t)k * r + k];
                __syncthreads();
            }
            for (int k = r - 1; k >= 0; --k) {   // L^T w = z (unit diagonal; w in a)
                double t = 0.0;
                for (int l = k + 1 + tid; l < r; l += kFThreads) t += M[(size_t)l * r + k] * a[l];
                t = block_sum(t, red);
                if (tid == 0) a[k] -= t;
                __syncthreads();
            }
            // a <- P^T w: the w entry at position k belongs to original row piv[k]
            for (int k = tid; k < r; k += kFThreads) u0[k] = a[k];
            __syncthreads();
            for (int k = tid; k < r; k += kFThreads) a[piv[k]] = u0[k];
            __syncthreads();
        }
        if constexpr (FF_) {
            // the pivot points' own terms first, then gs / gt hold c and a as
            // float-float pairs for the point loops
            for (int k = tid; k < r; k += kFThreads) gadd(A.G, tp[k], -0.5 * c[k], gt[k][0], gt[k][1], gt[k][2]);
            for (int k = tid; k < r; k += kFThreads) gadd(A.G, sp[k], 0.5 * a[k], gs[k][0], gs[k][1], gs[k][2]);
            __syncthreads();
            float2 *cf = reinterpret_cast<float2 *>(&gs[0][0]), *af = reinterpret_cast<float2 *>(&gt[0][0]);
            for (int k = tid; k < r; k += kFThreads) {
                const FF x = ff_from_double(c[k]), y = ff_from_double(a[k]);
                cf[k] = make_float2(x.h, x.l);
                af[k] = make_float2(y.h, y.l);
            }
            __syncthreads();
            // first term: q_X^T dK(X,tau) c
            for (int i = x0 + tid; i < x0 + m; i += kFThreads) {
                const float4 hi = A.ph[i], li = A.pl[i];
                FF g[3] = {FF{0.f, 0.f}, FF{0.f, 0.f}, FF{0.f, 0.f}};
                for (int k = 0; k < r; ++k) {
                    const int pt = tp[k];
                    FF f, fr, d[3];
                    ff_kernel_grad(A.kind, hi, li, A.ph[pt], A.pl[pt], f, fr, d);
                    const FF w = ff_mul(fr, FF{cf[k].x, cf[k].y});
#pragma unroll
                    for (int q = 0; q < 3; ++q) g[q] = ff_fma_acc(g[q], w, d[q]);
                }
                gadd(A.G, i, 0.5 * A.qs[i], ff_to_double(g[0]), ff_to_double(g[1]), ff_to_double(g[2]));
            }
            // second term: a^T dK(sigma,Y) q_Y
            for (int j = y0 + tid; j < y0 + n; j += kFThreads) {
                const float4 hj = A.ph[j], lj = A.pl[j];
                FF g[3] = {FF{0.f, 0.f}, FF{0.f, 0.f}, FF{0.f, 0.f}};
                for (int k = 0; k < r; ++k) {
                    const int ps = sp[k];
                    FF f, fr, d[3];
                    ff_kernel_grad(A.kind, A.ph[ps], A.pl[ps], hj, lj, f, fr, d);
                    const FF w = ff_mul(fr, FF{af[k].x, af[k].y});
#pragma unroll
                    for (int q = 0; q < 3; ++q) g[q] = ff_fma_acc(g[q], w, d[q]);
                }
                gadd(A.G, j, -0.5 * A.qs[j], ff_to_double(g[0]), ff_to_double(g[1]), ff_to_double(g[2]));
            }
            // third term: - a^T dM c
            for (int k = tid; k < r; k += kFThreads) {
                const float4 hs = A.ph[sp[k]], ls = A.pl[sp[k]], ht = A.ph[tp[k]], lt = A.pl[tp[k]];
                FF g[3] = {FF{0.f, 0.f}, FF{0.f, 0.f}, FF{0.f, 0.f}}, h[3] = {FF{0.f, 0.f}, FF{0.f, 0.f}, FF{0.f, 0.f}};
                for (int l = 0; l < r; ++l) {
                    FF f, fr, d[3];
                    ff_kernel_grad(A.kind, hs, ls, A.ph[tp[l]], A.pl[tp[l]], f, fr, d);
                    const FF w = ff_mul(fr, FF{cf[l].x, cf[l].y});
#pragma unroll
                    for (int q = 0; q < 3; ++q) g[q] = ff_fma_acc(g[q], w, d[q]);
                    ff_kernel_grad(A.kind, A.ph[sp[l]], A.pl[sp[l]], ht, lt, f, fr, d);
                    const FF w1 = ff_mul(fr, FF{af[l].x, af[l].y});
#pragma unroll
                    for (int q = 0; q < 3; ++q) h[q] = ff_fma_acc(h[q], w1, d[q]);
                }
                gadd(A.G, sp[k], -0.5 * a[k], ff_to_double(g[0]), ff_to_double(g[1]), ff_to_double(g[2]));
                gadd(A.G, tp[k], 0.5 * c[k], ff_to_double(h[0]), ff_to_double(h[1]), ff_to_double(h[2]));
            }
        } else {
            // first term: q_X^T dK(X,tau) c (pivots in pairs: two independent chains)
            for (int i = x0 + tid; i < x0 + m; i += kFThreads) {
                T gx = 0, gy = 0, gz = 0, fx = 0, fy = 0, fz = 0;
                int k = 0;
                for (; k + 1 < r; k += 2) {
                    double dx, dy, dz, ex, ey, ez, fr, fr1;
                    pdiff(A, i, tp[k], dx, dy, dz);
                    pdiff(A, i, tp[k + 1], ex, ey, ez);
                    kval_fr(A.kind, A.kappa, fma(dz, dz, fma(dy, dy, dx * dx)), fr);
                    kval_fr(A.kind, A.kappa, fma(ez, ez, fma(ey, ey, ex * ex)), fr1);
                    const T w = (T)c[k] * fr, w1 = (T)c[k + 1] * fr1;
                    gx = fma(w, dx, gx); gy = fma(w, dy, gy); gz = fma(w, dz, gz);
                    fx = fma(w1, ex, fx); fy = fma(w1, ey, fy); fz = fma(w1, ez, fz);
                }
                if (k < r) {
                    double dx, dy, dz, fr;
                    pdiff(A, i, tp[k], dx, dy, dz);
                    kval_fr(A.kind, A.kappa, fma(dz, dz, fma(dy, dy, dx * dx)), fr);
                    const T w = (T)c[k] * fr;
                    gx = fma(w, dx, gx); gy = fma(w, dy, gy); gz = fma(w, dz, gz);
                }
                gadd(A.G, i, 0.5 * A.qs[i], gx + fx, gy + fy, gz + fz);
            }
            for (int k = tid; k < r; k += kFThreads) gadd(A.G, tp[k], -0.5 * c[k], gt[k][0], gt[k][1], gt[k][2]);
            // second term: a^T dK(sigma,Y) q_Y
            for (int k = tid; k < r; k += kFThreads) gadd(A.G, sp[k], 0.5 * a[k], gs[k][0], gs[k][1], gs[k][2]);
            for (int j = y0 + tid; j < y0 + n; j += kFThreads) {
                T gx = 0, gy = 0, gz = 0, fx = 0, fy = 0, fz = 0;
                int k = 0;
                for (; k + 1 < r; k += 2) {
                    double dx, dy, dz, ex, ey, ez, fr, fr1;
                    pdiff(A, sp[k], j, dx, dy, dz);
                    pdiff(A, sp[k + 1], j, ex, ey, ez);
                    kval_fr(A.kind, A.kappa, fma(dz, dz, fma(dy, dy, dx * dx)), fr);
                    kval_fr(A.kind, A.kappa, fma(ez, ez, fma(ey, ey, ex * ex)), fr1);
                    const T w = (T)a[k] * fr, w1 = (T)a[k + 1] * fr1;
                    gx = fma(w, dx, gx); gy = fma(w, dy, gy); gz = fma(w, dz, gz);
                    fx = fma(w1, ex, fx); fy = fma(w1, ey, fy); fz = fma(w1, ez, fz);
                }
                if (k < r) {
                    double dx, dy, dz, fr;
                    pdiff(A, sp[k], j, dx, dy, dz);
                    kval_fr(A.kind, A.kappa, fma(dz, dz, fma(dy, dy, dx * dx)), fr);
                    const T w = (T)a[k] * fr;
                    gx = fma(w, dx, gx); gy = fma(w, dy, gy); gz = fma(w, dz, gz);
                }
                gadd(A.G, j, -0.5 * A.qs[j], gx + fx, gy + fy, gz + fz);
            }
        }
        // third term: - a^T dM c (FP64; float-float above for FF_)
        for (int k = tid; k < r && !FF_; k += kFThreads) {
            double gx = 0.0, gy = 0.0, gz = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
            for (int l = 0; l < r; ++l) {
                double dx, dy, dz, ex, ey, ez, fr, fr1;
                pdiff(A, sp[k], tp[l], dx, dy, dz);
                pdiff(A, sp[l], tp[k], ex, ey, ez);
                kval_fr(A.kind, A.kappa, fma(dz, dz, fma(dy, dy, dx * dx)), fr);
                kval_fr(A.kind, A.kappa, fma(ez, ez, fma(ey, ey, ex * ex)), fr1);
                const double w = c[l] * fr, w1 = a[l] * fr1;
                gx = fma(w, dx, gx); gy = fma(w, dy, gy); gz = fma(w, dz, gz);
                fx = fma(w1, ex, fx); fy = fma(w1, ey, fy); fz = fma(w1, ez, fz);
            }
            gadd(A.G, sp[k], -0.5 * a[k], gx, gy, gz);
            gadd(A.G, tp[k], 0.5 * c[k], fx, fy, fz);
        }
        __syncthreads();
    }
}

__global__ void k_forces_out(const double *__restrict__ G, const int *__restrict__ perm, int64_t n,
                             double *__restrict__ F) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t o = perm[s];
    F[3 * o] = -G[3 * s];
    F[3 * o + 1] = -G[3 * s + 1];
    F[3 * o + 2] = -G[3 * s + 2];
}

__global__ void k_sum_parts(const double *__restrict__ part, int64_t np, double *__restrict__ out, int nout) {
    // out[b] = sum of one contiguous share of part (fixed order)
    __shared__ double red[256];
    const int64_t per = (np + nout - 1) / nout;
    const int64_t lo = (int64_t)blockIdx.x * per, hi = min(np, lo + per);
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += 256) acc += part[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

unsigned gn(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

void forces(Handle &h, const void *q, double *E, double *F, cudaStream_t s) {
    int dev = 0, sms = 0;
    H3D_CUDA(cudaGetDevice(&dev));
    H3D_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // CTAs per SM: up to kFarCtasMax while their arrays fit the SM's shared memory
    const size_t fsm = far_smem(std::max(1, h.max_rank));
    const int far_ctas = (int)std::max<size_t>(1, std::min<size_t>(kFarCtasMax, (200u << 10) / (fsm + 1024)));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(h.nblk, (int64_t)far_ctas * sms));
    const int64_t nparts = h.nleaf + h.nblk;
    const bool fp32 = h.prec != H3D_FP64;
    if (!h.fG) {   // scratch kept by the handle
        H3D_CUDA(cudaStreamSynchronize(s));
        const size_t n1 = (size_t)std::max<int64_t>(h.N, 1), mr = (size_t)std::max(1, h.max_rank);
        void *ph = nullptr, *pl = nullptr;
        alloc_all(h.mem, {{(void **)&h.fqs, n1 * sizeof(double)},
                          {(void **)&h.fE, ((size_t)std::max<int64_t>(nparts, 1) + 1024) * sizeof(double)},
                          {(void **)&h.fM, (size_t)grid * mr * mr * sizeof(double)},
                          {(void **)&h.fctr, sizeof(int)},
                          {&ph, fp32 ? n1 * sizeof(float4) : 16},
                          {&pl, fp32 ? n1 * sizeof(float4) : 16},
                          {(void **)&h.fG, n1 * 3 * sizeof(double)}});   // fG last: it marks the scratch as made
        if (fp32) {
            h.fph = static_cast<float4 *>(ph);
            h.fpl = static_cast<float4 *>(pl);
        }
    }
    const int64_t N = h.N;
    if (fp32)
        k_charges_sorted<float><<<gn(N, 256), 256, 0, s>>>((const float *)q, h.perm, h.px, h.py, h.pz, N, h.fqs,
                                                            h.fph, h.fpl);
    else
        k_charges_sorted<double><<<gn(N, 256), 256, 0, s>>>((const double *)q, h.perm, h.px, h.py, h.pz, N, h.fqs,
                                                             nullptr, nullptr);
    ForceArgs A{};
    A.kind = h.kernel;
    A.kappa = h.kappa;
    A.px = h.px; A.py = h.py; A.pz = h.pz;
    A.ph = h.fph; A.pl = h.fpl;
    A.qs = h.fqs;
    A.G = h.fG;
    A.offL = h.box_off[h.L];
    A.nleaf = h.nleaf;
    A.box_start = h.box_start; A.box_end = h.box_end;
    A.near_ptr = h.near_ptr; A.near_src = h.near_src;
    A.nblk = h.nblk;
    A.blk_tgt = h.blk_tgt; A.blk_src = h.blk_src; A.rank = h.rank; A.sigma = h.sigma; A.tau = h.tau;
    A.piv_off = h.piv_off;
    A.Mscr = h.fM;
    A.mr = std::max(1, h.max_rank);
    A.Epart = h.fE + 1024;
    A.next = h.fctr;
    // the near kernel writes every point's gradient (each point lies in one leaf),
    // the far kernel then adds to it
    if (fp32)
        k_force_near<float><<<h.nleaf, kFThreads, 0, s>>>(A);
    else
        k_force_near<double><<<h.nleaf, kFThreads, 0, s>>>(A);
    if (h.nblk > 0) {
        H3D_CUDA(cudaMemsetAsync(h.fctr, 0, sizeof(int), s));
        if (fp32 && ff_kernel_supported(h.kernel)) k_force_far<true><<<grid, kFThreads, fsm, s>>>(A);
        else k_force_far<false><<<grid, kFThreads, fsm, s>>>(A);
    }
    k_forces_out<<<gn(N, 256), 256, 0, s>>>(h.fG, h.perm, N, F);
    const int nout = (int)std::min<int64_t>(1024, std::max<int64_t>(1, nparts));
    k_sum_parts<<<nout, 256, 0, s>>>(h.fE + 1024, nparts, h.fE, nout);
    k_sum_parts<<<1, 256, 0, s>>>(h.fE, nout, E, 1);
    H3D_LAUNCH_CHECK();
}

}  // namespace h3d
