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
// recomputed (nothing is stored), in FP64; M is factored by Gaussian elimination
// with partial pivoting in FP64.  Far-field contributions reach the points
// through FP64 atomic additions; the energy is reduced in a fixed order.
#include "h3d_internal.cuh"

namespace h3d {
namespace {

constexpr int kFThreads = 128;
constexpr int kFWarps = kFThreads / 32;

// K(a, b) and dK/da for a - b = (dx, dy, dz)
__device__ __forceinline__ double kval_grad(int kind, double kappa, double dx, double dy, double dz, double &gx,
                                            double &gy, double &gz) {
    const double d2 = dx * dx + dy * dy + dz * dz;
    if (d2 == 0.0) {
        gx = gy = gz = 0.0;
        return 0.0;
    }
    const double r = sqrt(d2), ir = 1.0 / r;
    double f, fp;
    switch (kind) {
    case H3D_LAPLACE: f = H3D_INV4PI * ir; fp = -f * ir; break;
    case H3D_YUKAWA: {
        const double e = exp(-kappa * r);
        f = H3D_INV4PI * e * ir;
        fp = -f * (1.0 + kappa * r) * ir;
        break;
    }
    case H3D_INV_R4: f = 1.0 / (d2 * d2); fp = -4.0 * f * ir; break;
    default: {
        double sn, cs;
        sincos(r, &sn, &cs);
        f = cs * ir;
        fp = -(r * sn + cs) * ir * ir;
    }
    }
    const double s = fp * ir;
    gx = s * dx;
    gy = s * dy;
    gz = s * dz;
    return f;
}

__device__ __forceinline__ double kval(int kind, double kappa, double dx, double dy, double dz) {
    double gx, gy, gz;
    return kval_grad(kind, kappa, dx, dy, dz, gx, gy, gz);
}

struct ForceArgs {
    int kind;
    double kappa;
    const double *px, *py, *pz;
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
};

template <class T>
__global__ void k_charges_sorted(const T *__restrict__ q, const int *__restrict__ perm, int64_t n,
                                 double *__restrict__ qs) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) qs[s] = (double)q[perm[s]];
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

// near field: every point of a leaf against every point of its near leaves
__global__ void __launch_bounds__(kFThreads) k_force_near(ForceArgs A) {
    __shared__ double red[kFWarps];
    const int z = blockIdx.x;
    const int Zg = (int)(A.offL + z);
    const int x0 = A.box_start[Zg], x1 = A.box_end[Zg];
    double e = 0.0;
    for (int i = x0 + threadIdx.x; i < x1; i += kFThreads) {
        const double xi = A.px[i], yi = A.py[i], zi = A.pz[i], qi = A.qs[i];
        double ei = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int p = A.near_ptr[z]; p < A.near_ptr[z + 1]; ++p) {
            const int Sg = (int)(A.offL + A.near_src[p]);
            for (int j = A.box_start[Sg]; j < A.box_end[Sg]; ++j) {
                if (j == i) continue;
                double hx, hy, hz;
                const double k = kval_grad(A.kind, A.kappa, xi - A.px[j], yi - A.py[j], zi - A.pz[j], hx, hy, hz);
                const double w = qi * A.qs[j];
                ei += A.qs[j] * k;
                gx += w * hx;
                gy += w * hy;
                gz += w * hz;
            }
        }
        e += 0.5 * qi * ei;
        A.G[3 * (int64_t)i] = gx;
        A.G[3 * (int64_t)i + 1] = gy;
        A.G[3 * (int64_t)i + 2] = gz;
    }
    const double t = block_sum(e, red);
    if (threadIdx.x == 0) A.Epart[z] = t;
}

__device__ __forceinline__ void gadd(double *G, int p, double s, double gx, double gy, double gz) {
    atomicAdd(G + 3 * (int64_t)p, s * gx);
    atomicAdd(G + 3 * (int64_t)p + 1, s * gy);
    atomicAdd(G + 3 * (int64_t)p + 2, s * gz);
}

// far field: one block at a time per CTA (grid-stride), M in this CTA's scratch
__global__ void __launch_bounds__(kFThreads) k_force_far(ForceArgs A) {
    __shared__ int sp[kMaxRank], tp[kMaxRank], piv[kMaxRank];
    __shared__ double c[kMaxRank], a[kMaxRank], u0[kMaxRank];
    __shared__ double red[kFWarps];
    __shared__ int pmax;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    double *M = A.Mscr + (size_t)blockIdx.x * A.mr * A.mr;
    for (int64_t b = blockIdx.x; b < A.nblk; b += gridDim.x) {
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
        // s = K(sigma, Y) q_Y -> c,  u = K(X, tau)^T q_X -> a (one warp per pivot)
        for (int k = warp; k < r; k += kFWarps) {
            const int ps = sp[k], pt = tp[k];
            double sv = 0.0, uv = 0.0;
            for (int j = y0 + lane; j < y0 + n; j += 32)
                sv += kval(A.kind, A.kappa, A.px[ps] - A.px[j], A.py[ps] - A.py[j], A.pz[ps] - A.pz[j]) * A.qs[j];
            for (int i = x0 + lane; i < x0 + m; i += 32)
                uv += A.qs[i] * kval(A.kind, A.kappa, A.px[i] - A.px[pt], A.py[i] - A.py[pt], A.pz[i] - A.pz[pt]);
            for (int o = 16; o > 0; o >>= 1) {
                sv += __shfl_xor_sync(0xffffffffu, sv, o);
                uv += __shfl_xor_sync(0xffffffffu, uv, o);
            }
            if (lane == 0) {
                c[k] = sv;
                a[k] = uv;
                u0[k] = uv;
            }
        }
        // M = K(sigma, tau), row-major r x r
        for (int e = tid; e < r * r; e += kFThreads) {
            const int k = e / r, l = e - k * r;
            const int ps = sp[k], pt = tp[l];
            M[e] = kval(A.kind, A.kappa, A.px[ps] - A.px[pt], A.py[ps] - A.py[pt], A.pz[ps] - A.pz[pt]);
        }
        for (int k = tid; k < r; k += kFThreads) piv[k] = k;
        __syncthreads();
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
        // energy 1/2 u^T c (u recomputed: u0 was reused)
        {
            double e = 0.0;
            for (int k = warp; k < r; k += kFWarps) {
                const int pt = tp[k];
                double uv = 0.0;
                for (int i = x0 + lane; i < x0 + m; i += 32)
                    uv += A.qs[i] * kval(A.kind, A.kappa, A.px[i] - A.px[pt], A.py[i] - A.py[pt], A.pz[i] - A.pz[pt]);
                for (int o = 16; o > 0; o >>= 1) uv += __shfl_xor_sync(0xffffffffu, uv, o);
                if (lane == 0) e += 0.5 * uv * c[k];
            }
            e = block_sum(e, red);
            if (tid == 0) A.Epart[A.nleaf + b] = e;
        }
        // first term: q_X^T dK(X,tau) c
        for (int i = x0 + tid; i < x0 + m; i += kFThreads) {
            double gx = 0.0, gy = 0.0, gz = 0.0;
            for (int k = 0; k < r; ++k) {
                const int pt = tp[k];
                double hx, hy, hz;
                kval_grad(A.kind, A.kappa, A.px[i] - A.px[pt], A.py[i] - A.py[pt], A.pz[i] - A.pz[pt], hx, hy, hz);
                gx += c[k] * hx;
                gy += c[k] * hy;
                gz += c[k] * hz;
            }
            gadd(A.G, i, 0.5 * A.qs[i], gx, gy, gz);
        }
        for (int k = warp; k < r; k += kFWarps) {
            const int pt = tp[k];
            double gx = 0.0, gy = 0.0, gz = 0.0;
            for (int i = x0 + lane; i < x0 + m; i += 32) {
                double hx, hy, hz;
                kval_grad(A.kind, A.kappa, A.px[i] - A.px[pt], A.py[i] - A.py[pt], A.pz[i] - A.pz[pt], hx, hy, hz);
                gx += A.qs[i] * hx;
                gy += A.qs[i] * hy;
                gz += A.qs[i] * hz;
            }
            for (int o = 16; o > 0; o >>= 1) {
                gx += __shfl_xor_sync(0xffffffffu, gx, o);
                gy += __shfl_xor_sync(0xffffffffu, gy, o);
                gz += __shfl_xor_sync(0xffffffffu, gz, o);
            }
            if (lane == 0) gadd(A.G, pt, -0.5 * c[k], gx, gy, gz);
        }
        // second term: a^T dK(sigma,Y) q_Y
        for (int k = warp; k < r; k += kFWarps) {
            const int ps = sp[k];
            double gx = 0.0, gy = 0.0, gz = 0.0;
            for (int j = y0 + lane; j < y0 + n; j += 32) {
                double hx, hy, hz;
                kval_grad(A.kind, A.kappa, A.px[ps] - A.px[j], A.py[ps] - A.py[j], A.pz[ps] - A.pz[j], hx, hy, hz);
                gx += A.qs[j] * hx;
                gy += A.qs[j] * hy;
                gz += A.qs[j] * hz;
            }
            for (int o = 16; o > 0; o >>= 1) {
                gx += __shfl_xor_sync(0xffffffffu, gx, o);
                gy += __shfl_xor_sync(0xffffffffu, gy, o);
                gz += __shfl_xor_sync(0xffffffffu, gz, o);
            }
            if (lane == 0) gadd(A.G, ps, 0.5 * a[k], gx, gy, gz);
        }
        for (int j = y0 + tid; j < y0 + n; j += kFThreads) {
            double gx = 0.0, gy = 0.0, gz = 0.0;
            for (int k = 0; k < r; ++k) {
                const int ps = sp[k];
                double hx, hy, hz;
                kval_grad(A.kind, A.kappa, A.px[ps] - A.px[j], A.py[ps] - A.py[j], A.pz[ps] - A.pz[j], hx, hy, hz);
                gx += a[k] * hx;
                gy += a[k] * hy;
                gz += a[k] * hz;
            }
            gadd(A.G, j, -0.5 * A.qs[j], gx, gy, gz);
        }
        // third term: - a^T dM c
        for (int k = tid; k < r; k += kFThreads) {
            const int ps = sp[k];
            double gx = 0.0, gy = 0.0, gz = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
            for (int l = 0; l < r; ++l) {
                const int pt = tp[l];
                double hx, hy, hz;
                kval_grad(A.kind, A.kappa, A.px[ps] - A.px[pt], A.py[ps] - A.py[pt], A.pz[ps] - A.pz[pt], hx, hy, hz);
                gx += c[l] * hx;
                gy += c[l] * hy;
                gz += c[l] * hz;
                // entry (l, k) of the same sums for the column-pivot side
                const int ps2 = sp[l], pt2 = tp[k];
                kval_grad(A.kind, A.kappa, A.px[ps2] - A.px[pt2], A.py[ps2] - A.py[pt2], A.pz[ps2] - A.pz[pt2], hx, hy,
                          hz);
                fx += a[l] * hx;
                fy += a[l] * hy;
                fz += a[l] * hz;
            }
            gadd(A.G, ps, -0.5 * a[k], gx, gy, gz);
            gadd(A.G, tp[k], 0.5 * c[k], fx, fy, fz);
        }
        __syncthreads();
    }
}

template <class T>
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
    // out[b] = sum of part[b*per ... ]: fixed blocked order
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
    constexpr int kFarCtas = 2;   // per SM
    int dev = 0, sms = 0;
    H3D_CUDA(cudaGetDevice(&dev));
    H3D_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(h.nblk, (int64_t)kFarCtas * sms));
    const int64_t nparts = h.nleaf + h.nblk;
    if (!h.fG) {   // scratch kept by the handle
        H3D_CUDA(cudaStreamSynchronize(s));
        h.fqs = h.mem.get<double>((size_t)std::max<int64_t>(h.N, 1));
        h.fG = h.mem.get<double>((size_t)std::max<int64_t>(h.N, 1) * 3);
        h.fE = h.mem.get<double>((size_t)std::max<int64_t>(nparts, 1) + 1024);
        h.fM = h.mem.get<double>((size_t)grid * std::max(1, h.max_rank) * std::max(1, h.max_rank));
    }
    const int64_t N = h.N;
    if (h.prec == H3D_FP64)
        k_charges_sorted<double><<<gn(N, 256), 256, 0, s>>>((const double *)q, h.perm, N, h.fqs);
    else
        k_charges_sorted<float><<<gn(N, 256), 256, 0, s>>>((const float *)q, h.perm, N, h.fqs);
    ForceArgs A{};
    A.kind = h.kernel;
    A.kappa = h.kappa;
    A.px = h.px; A.py = h.py; A.pz = h.pz;
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
    k_force_near<<<h.nleaf, kFThreads, 0, s>>>(A);   // writes G (every point lies in one leaf)
    if (h.nblk > 0) k_force_far<<<grid, kFThreads, 0, s>>>(A);
    k_forces_out<double><<<gn(N, 256), 256, 0, s>>>(h.fG, h.perm, N, F);
    const int nout = (int)std::min<int64_t>(1024, std::max<int64_t>(1, nparts));
    k_sum_parts<<<nout, 256, 0, s>>>(h.fE + 1024, nparts, h.fE, nout);
    k_sum_parts<<<1, 256, 0, s>>>(h.fE, nout, E, 1);
    H3D_LAUNCH_CHECK();
}

}  // namespace h3d
