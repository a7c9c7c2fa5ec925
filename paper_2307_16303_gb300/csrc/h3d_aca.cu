// h3d_aca.cu -- batched partially pivoted ACA of every admissible block
// (Sec. 4.1, Eq. prank, Alg. 1 inner loop) and packing of the factors into the
// layout streamed by the product.
//
// ACA, per block X x Y (rows = target points, columns = source points):
//   the first pivot row is local row 0; the residual of pivot row i is
//   K(i,:) - sum_{l<k} U(i,l) V(:,l) accumulated with fma in l order; the
//   column pivot j* maximises |residual| over unused columns (ties: smallest
//   index); a vanishing residual row is skipped for the smallest unused row;
//   V(:,k) = residual / residual(j*); U(:,k) = K(:,j*) - sum_{l<k} V(j*,l) U(:,l);
//   the next row pivot maximises |U(:,k)| over unused rows; the Frobenius norm
//   of the approximant is updated with its cross terms and the iteration stops
//   when |U(:,k)| |V(:,k)| <= tol |S_k|_F or at min(m, n, rank_cap).
// U V^T equals K(X,tau) K(sigma,tau)^{-1} K(sigma,Y) of Eq. prank; the product
// streams U and V instead of re-forming them from the pivots (memory permits
// it on a 288 GB GPU at the sizes of Sec. 5.1).
//
// All of it is FP64 with explicitly rounded operations, so the residuals (and
// hence the pivots) are reproducible bit for bit by a plain C evaluation; only
// the order of the norm sums differs, which can move a borderline stop.
//
// Two passes: pass 1 searches pivots with scratch sized by min(m, n, rank_cap);
// pass 2 re-forms U and V from the frozen pivots (same arithmetic, same bits)
// with scratch sized by the rank, and converts them into the final layout.
#include <algorithm>
#include <climits>

#include "h3d_internal.cuh"

namespace h3d {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kSmallMax = 512;  // max(m, n) up to this: one warp per block
constexpr int kChunk = 8;       // cross-term dot products reduced per pass

struct AcaJob {
    int blk, m, n, cap;     // cap: search limit (pass 1) or frozen rank (pass 2)
    int xs, ys;             // first sorted point of X and Y
    int64_t uoff, voff;     // scratch offsets (doubles): U m x cap, V n x cap, column-major
    int64_t foff;           // flag offset (bytes): m row flags then n column flags
    int64_t poff;           // pivot offset: pass 1 scratch slot / pass 2 final offset
};

struct AcaArgs {
    const double *px, *py, *pz;
    int kind;
    double kappa, tol;
    double *scratch;
    unsigned char *flags;
    int *sig, *tau;         // pivots (pass 1: scratch slots; pass 2: final arrays, read)
    int *rank;              // per block (written by pass 1)
    int *err;
};

// ----------------------------------------------------------------------------
// cooperative groups of NT threads: a warp (NT = 32) or a whole CTA.
template <int NT>
struct Grp {
    double *red;  // kWarps * (kChunk * 2 + 2) doubles for NT > 32
    int *redi;    // kWarps * 2 ints
    __device__ __forceinline__ int rank() const { return NT == 32 ? (threadIdx.x & 31) : threadIdx.x; }
    __device__ __forceinline__ void sync() const {
        if (NT == 32) __syncwarp(); else __syncthreads();
    }
    template <int NV>
    __device__ __forceinline__ void sum(double (&v)[NV]) const {
#pragma unroll
        for (int q = 0; q < NV; ++q)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        if (NT > 32) {
            const int w = threadIdx.x >> 5;
            if ((threadIdx.x & 31) == 0)
#pragma unroll
                for (int q = 0; q < NV; ++q) red[w * NV + q] = v[q];
            __syncthreads();
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                double s = 0.0;
                for (int u = 0; u < NT / 32; ++u) s += red[u * NV + q];
                v[q] = s;
            }
            __syncthreads();
        }
    }
    // largest value, ties to the smallest index
    __device__ __forceinline__ void argmax(double &v, int &i) const {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, v, o);
            int oi = __shfl_xor_sync(0xffffffffu, i, o);
            if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
        }
        if (NT > 32) {
            const int w = threadIdx.x >> 5;
            if ((threadIdx.x & 31) == 0) { red[w] = v; redi[w] = i; }
            __syncthreads();
            v = red[0]; i = redi[0];
            for (int u = 1; u < NT / 32; ++u) {
                double ov = red[u]; int oi = redi[u];
                if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
            }
            __syncthreads();
        }
    }
    __device__ __forceinline__ int min_index(int i) const {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) i = min(i, __shfl_xor_sync(0xffffffffu, i, o));
        if (NT > 32) {
            const int w = threadIdx.x >> 5;
            if ((threadIdx.x & 31) == 0) redi[w] = i;
            __syncthreads();
            i = redi[0];
            for (int u = 1; u < NT / 32; ++u) i = min(i, redi[u]);
            __syncthreads();
        }
        return i;
    }
};

template <int NT, bool FROZEN>
__device__ void aca_block(const AcaJob &J, const AcaArgs &A, const Grp<NT> &g, double *rowbuf) {
    const int m = J.m, n = J.n, cap = J.cap;
    const int t0 = g.rank();
    double *U = A.scratch + J.uoff;
    double *V = A.scratch + J.voff;
    unsigned char *urow = FROZEN ? nullptr : A.flags + J.foff;
    unsigned char *ucol = FROZEN ? nullptr : urow + m;
    const double *Xx = A.px + J.xs, *Xy = A.py + J.xs, *Xz = A.pz + J.xs;
    const double *Yx = A.px + J.ys, *Yy = A.py + J.ys, *Yz = A.pz + J.ys;
    int *sig = A.sig + J.poff, *tau = A.tau + J.poff;

    if (!FROZEN) {
        for (int t = t0; t < m + n; t += NT) urow[t] = 0;
    }
    g.sync();
    int k = 0;
    int i = FROZEN ? (cap > 0 ? sig[0] : 0) : 0;
    double S2 = 0.0;
    bool converged = false;
    for (;;) {
        if (k == cap) break;
        g.sync();  // nobody still reads rowbuf from the previous step
        // ---- residual of row i -> V(:,k)
        for (int l = t0; l < k; l += NT) rowbuf[l] = U[(int64_t)l * m + i];
        g.sync();
        const double xi = Xx[i], yi = Xy[i], zi = Xz[i];
        double best = -1.0;
        int bj = INT_MAX;
        double *Vk = V + (int64_t)k * n;
        for (int j = t0; j < n; j += NT) {
            double r = kernel_exact(A.kind, A.kappa, xi, yi, zi, Yx[j], Yy[j], Yz[j]);
            for (int l = 0; l < k; ++l) r = __fma_rn(-rowbuf[l], V[(int64_t)l * n + j], r);
            Vk[j] = r;
            if (!FROZEN) {
                const double a = fabs(r);
                if (!ucol[j] && a > best) { best = a; bj = j; }
            }
        }
        int jstar;
        if (FROZEN) {
            jstar = tau[k];
        } else {
            g.argmax(best, bj);
            if (t0 == 0) urow[i] = 1;
            if (bj == INT_MAX || best == 0.0) {
                g.sync();
                int cand = INT_MAX;
                for (int t = t0; t < m; t += NT)
                    if (!urow[t]) { cand = t; break; }
                cand = g.min_index(cand);
                if (cand == INT_MAX) { converged = true; break; }
                i = cand;
                continue;
            }
            jstar = bj;
        }
        g.sync();
        const double delta = Vk[jstar];
        g.sync();
        for (int j = t0; j < n; j += NT) Vk[j] = __ddiv_rn(Vk[j], delta);
        if (!FROZEN && t0 == 0) ucol[jstar] = 1;
        // ---- residual of column jstar -> U(:,k)
        for (int l = t0; l < k; l += NT) rowbuf[l] = V[(int64_t)l * n + jstar];
        g.sync();
        const double xj = Yx[jstar], yj = Yy[jstar], zj = Yz[jstar];
        double *Uk = U + (int64_t)k * m;
        double bu = -1.0;
        int bi = INT_MAX;
        for (int t = t0; t < m; t += NT) {
            double u = kernel_exact(A.kind, A.kappa, Xx[t], Xy[t], Xz[t], xj, yj, zj);
            for (int l = 0; l < k; ++l) u = __fma_rn(-rowbuf[l], U[(int64_t)l * m + t], u);
            Uk[t] = u;
            if (!FROZEN) {
                const double a = fabs(u);
                if (!urow[t] && a > bu) { bu = a; bi = t; }
            }
        }
        if (!FROZEN && t0 == 0) { sig[k] = i; tau[k] = jstar; }
        ++k;
        if (FROZEN) {
            if (k < cap) i = sig[k];
            g.sync();
            continue;
        }
        g.sync();
        // ---- stopping test: |S_k|_F^2 = |S_{k-1}|^2 + 2 sum_l (u_l.u_k)(v_l.v_k) + |u_k|^2 |v_k|^2
        double nrm[2] = {0.0, 0.0};
        for (int t = t0; t < m; t += NT) nrm[0] += Uk[t] * Uk[t];
        for (int j = t0; j < n; j += NT) nrm[1] += Vk[j] * Vk[j];
        g.template sum<2>(nrm);
        double cross = 0.0;
        for (int l0 = 0; l0 < k - 1; l0 += kChunk) {
            double d[2 * kChunk];
#pragma unroll
            for (int q = 0; q < 2 * kChunk; ++q) d[q] = 0.0;
            const int lc = min(kChunk, k - 1 - l0);
            for (int t = t0; t < m; t += NT) {
                const double u = Uk[t];
#pragma unroll
                for (int q = 0; q < kChunk; ++q)
                    if (q < lc) d[q] += U[(int64_t)(l0 + q) * m + t] * u;
            }
            for (int j = t0; j < n; j += NT) {
                const double v = Vk[j];
#pragma unroll
                for (int q = 0; q < kChunk; ++q)
                    if (q < lc) d[kChunk + q] += V[(int64_t)(l0 + q) * n + j] * v;
            }
            g.template sum<2 * kChunk>(d);
            for (int q = 0; q < lc; ++q) cross += d[q] * d[kChunk + q];
        }
        S2 = S2 + 2.0 * cross + nrm[0] * nrm[1];
        if (S2 < 0.0) S2 = 0.0;
        if (sqrt(nrm[0]) * sqrt(nrm[1]) <= A.tol * sqrt(S2)) { converged = true; break; }
        g.argmax(bu, bi);
        if (bi == INT_MAX) { converged = true; break; }
        i = bi;
    }
    if (!FROZEN && t0 == 0) {
        A.rank[J.blk] = k;
        if (!converged && cap < min(m, n)) atomicOr(A.err, 1 << H3D_ERR_ACA_RANK);
    }
}

template <bool FROZEN>
__global__ void __launch_bounds__(kThreads) k_aca_warp(const AcaJob *__restrict__ jobs, int njobs, AcaArgs A,
                                                       int rowcap) {
    extern __shared__ double smem[];
    const int w = threadIdx.x >> 5;
    const int j = blockIdx.x * kWarps + w;
    if (j >= njobs) return;
    Grp<32> g{nullptr, nullptr};
    aca_block<32, FROZEN>(jobs[j], A, g, smem + (int64_t)w * rowcap);
}

template <bool FROZEN>
__global__ void __launch_bounds__(kThreads) k_aca_cta(const AcaJob *__restrict__ jobs, int njobs, AcaArgs A) {
    extern __shared__ double smem[];
    __shared__ double red[kWarps * (2 * kChunk + 2)];
    __shared__ int redi[kWarps * 2];
    if ((int)blockIdx.x >= njobs) return;
    Grp<kThreads> g{red, redi};
    aca_block<kThreads, FROZEN>(jobs[blockIdx.x], A, g, smem);
}

// ----------------------------------------------------------------------------
// layout kernels

// per box: R (sum of ranks over the target segment) and cu (prefix inside it)
__global__ void k_target_cols(const int64_t *__restrict__ tgt_ptr, const int *__restrict__ rank, int64_t nboxes,
                              int *__restrict__ R, int *__restrict__ cu) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nboxes) return;
    int acc = 0;
    for (int64_t b = tgt_ptr[g]; b < tgt_ptr[g + 1]; ++b) {
        cu[b] = acc;
        acc += rank[b];
    }
    R[g] = acc;
}

// per box Y: columns of the blocks whose source is Y, in order of their target
// (the partners of Y's own target segment, which is sorted by source).
__global__ void k_source_cols(const int64_t *__restrict__ tgt_ptr, const int *__restrict__ partner,
                              const int *__restrict__ rank, int64_t nboxes, int vw, int *__restrict__ Rv,
                              int *__restrict__ ldv, int *__restrict__ cv, int *__restrict__ err) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nboxes) return;
    int acc = 0;
    for (int64_t b = tgt_ptr[g]; b < tgt_ptr[g + 1]; ++b) {
        const int p = partner[b];
        if (p < 0) {  // the lists are symmetric by construction; never expected
            atomicOr(err, 1 << H3D_ERR_STATE);
            continue;
        }
        cv[p] = acc;
        acc += rank[p];
    }
    Rv[g] = acc;
    ldv[g] = (int)round_up(acc, vw);
}

__global__ void k_box_sizes(const int *__restrict__ box_start, const int *__restrict__ box_end,
                            const int *__restrict__ R, const int *__restrict__ ldv,
                            const int *__restrict__ leaf_lo, const int *__restrict__ leaf_hi,
                            const int64_t *__restrict__ lp, int64_t nboxes, int64_t *__restrict__ usz,
                            int64_t *__restrict__ vsz) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nboxes) return;
    usz[g] = (int64_t)R[g] * (lp[leaf_hi[g]] - lp[leaf_lo[g]]);
    vsz[g] = (int64_t)(box_end[g] - box_start[g]) * ldv[g];
}

__global__ void k_leaf_ld(const int *__restrict__ box_start, const int *__restrict__ box_end, int64_t offL, int nleaf,
                          int vw, int *__restrict__ ld) {
    int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= nleaf) return;
    ld[z] = (int)round_up(box_end[offL + z] - box_start[offL + z], vw);
}

__global__ void k_map_v(const int *__restrict__ blk_src, const int *__restrict__ rank, const int *__restrict__ cv,
                        const int64_t *__restrict__ vcol0, const int64_t *__restrict__ tofs, int64_t nblk,
                        int64_t *__restrict__ map_v) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    const int64_t base = vcol0[blk_src[b]] + cv[b];
    for (int k = 0; k < rank[b]; ++k) map_v[base + k] = tofs[b] + k;
}

__global__ void k_copy_pivots(const AcaJob *__restrict__ jobs, int njobs, const int *__restrict__ rank,
                              const int64_t *__restrict__ piv_off, const int *__restrict__ ssig,
                              const int *__restrict__ stau, int *__restrict__ sig, int *__restrict__ tau) {
    int j = blockIdx.x;
    if (j >= njobs) return;
    const AcaJob J = jobs[j];
    const int r = rank[J.blk];
    const int64_t o = piv_off[J.blk];
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        sig[o + k] = ssig[J.poff + k];
        tau[o + k] = stau[J.poff + k];
    }
}

struct PackArgs {
    const int *tgt, *src, *cu, *cv, *R, *ldv, *leaf_lo, *leaf_ld, *point_leaf, *box_start;
    const int64_t *ubase, *vbase, *lp;
    int64_t offL;
};

template <class T>
__global__ void k_pack(const AcaJob *__restrict__ jobs, int njobs, const double *__restrict__ scratch, PackArgs P,
                       T *__restrict__ Uo, T *__restrict__ Vo) {
    const int j = blockIdx.x;
    if (j >= njobs) return;
    const AcaJob J = jobs[j];
    const int r = J.cap, m = J.m, n = J.n, b = J.blk;
    if (r == 0) return;
    const int A = P.tgt[b], Y = P.src[b];
    const int RA = P.R[A], cub = P.cu[b], cvb = P.cv[b], lvY = P.ldv[Y];
    const int64_t lp0 = P.lp[P.leaf_lo[A]];
    const double *Us = scratch + J.uoff, *Vs = scratch + J.voff;
    const int64_t ue = (int64_t)m * r, ve = (int64_t)n * r;
    for (int64_t e = threadIdx.x; e < ue; e += blockDim.x) {
        const int k = (int)(e / m), i = (int)(e - (int64_t)k * m);
        const int p = J.xs + i;
        const int z = P.point_leaf[p];
        const int iloc = p - P.box_start[P.offL + z];
        const int64_t panel = P.ubase[A] + (P.lp[z] - lp0) * RA;
        Uo[panel + (int64_t)(cub + k) * P.leaf_ld[z] + iloc] = (T)Us[e];
    }
    for (int64_t e = threadIdx.x; e < ve; e += blockDim.x) {
        const int k = (int)(e / n), jj = (int)(e - (int64_t)k * n);
        Vo[P.vbase[Y] + (int64_t)jj * lvY + cvb + k] = (T)Vs[e];
    }
}

// fused pairs of symmetric storage: U and V of the job's block into its slot of
// symF (column-major, leading dimensions ldm / ldn; padding cleared before,
// so padding rows hold zeros)
template <class T>
__global__ void k_pack_sym(const AcaJob *__restrict__ jobs, int njobs, const double *__restrict__ scratch,
                           const int *__restrict__ slot, const SymBlk *__restrict__ blks, T *__restrict__ F) {
    const int j = blockIdx.x;
    if (j >= njobs) return;
    const AcaJob J = jobs[j];
    const SymBlk B = blks[slot[J.blk]];
    const int r = J.cap, m = J.m, n = J.n;
    const double *Us = scratch + J.uoff, *Vs = scratch + J.voff;
    T *Fu = F + B.off, *Fv = F + B.off + (int64_t)r * B.ldm;
    for (int64_t e = threadIdx.x; e < (int64_t)m * r; e += blockDim.x) {
        const int k = (int)(e / m), i = (int)(e - (int64_t)k * m);
        Fu[(int64_t)k * B.ldm + i] = (T)Us[e];
    }
    for (int64_t e = threadIdx.x; e < (int64_t)n * r; e += blockDim.x) {
        const int k = (int)(e / n), i = (int)(e - (int64_t)k * n);
        Fv[(int64_t)k * B.ldn + i] = (T)Vs[e];
    }
}

unsigned gridn(int64_t n, int t = kThreads) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// Run one batch of jobs: small blocks one warp each, large ones a CTA each.
template <bool FROZEN>
void run_batch(const std::vector<AcaJob> &small, const std::vector<AcaJob> &large, int maxcap_small,
               int maxcap_large, const AcaArgs &A, AcaJob *d_jobs, cudaStream_t s) {
    if (!small.empty()) {
        H3D_CUDA(cudaMemcpyAsync(d_jobs, small.data(), small.size() * sizeof(AcaJob), cudaMemcpyHostToDevice, s));
        const int rowcap = std::max(1, maxcap_small);
        const size_t sm = (size_t)kWarps * rowcap * sizeof(double);
        k_aca_warp<FROZEN><<<gridn((int64_t)small.size(), kWarps), kThreads, sm, s>>>(d_jobs, (int)small.size(), A,
                                                                                       rowcap);
        H3D_LAUNCH_CHECK();
    }
    if (!large.empty()) {
        AcaJob *d2 = d_jobs + small.size();
        H3D_CUDA(cudaMemcpyAsync(d2, large.data(), large.size() * sizeof(AcaJob), cudaMemcpyHostToDevice, s));
        const size_t sm = (size_t)std::max(1, maxcap_large) * sizeof(double);
        k_aca_cta<FROZEN><<<(unsigned)large.size(), kThreads, sm, s>>>(d2, (int)large.size(), A);
        H3D_LAUNCH_CHECK();
    }
}

}  // namespace

namespace {

// host copies of the block geometry (for batch planning)
struct BlockGeometry {
    std::vector<int> tgt, src, bstart, bend;
    std::vector<int> partner;   // symmetric storage only: the block (src, tgt)
    int m(int64_t b) const { return bend[tgt[b]] - bstart[tgt[b]]; }
    int n(int64_t b) const { return bend[src[b]] - bstart[src[b]]; }
    // symmetric storage: the block of a pair that is not compressed itself
    bool mirror(int64_t b) const { return !partner.empty() && tgt[b] > src[b]; }
};

BlockGeometry block_geometry(const Handle &h, cudaStream_t s) {
    const int64_t nblk = h.nblk, nboxes = h.n_boxes;
    BlockGeometry g;
    g.tgt.resize(nblk);
    g.src.resize(nblk);
    if (h.symmetric()) {
        g.partner.resize(nblk);
        if (nblk > 0)
            H3D_CUDA(cudaMemcpyAsync(g.partner.data(), h.blk_partner, nblk * sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    g.bstart.resize(nboxes);
    g.bend.resize(nboxes);
    if (nblk > 0) {
        H3D_CUDA(cudaMemcpyAsync(g.tgt.data(), h.blk_tgt, nblk * sizeof(int), cudaMemcpyDeviceToHost, s));
        H3D_CUDA(cudaMemcpyAsync(g.src.data(), h.blk_src, nblk * sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    H3D_CUDA(cudaMemcpyAsync(g.bstart.data(), h.box_start, nboxes * sizeof(int), cudaMemcpyDeviceToHost, s));
    H3D_CUDA(cudaMemcpyAsync(g.bend.data(), h.box_end, nboxes * sizeof(int), cudaMemcpyDeviceToHost, s));
    H3D_CUDA(cudaStreamSynchronize(s));
    return g;
}

constexpr int64_t kMaxJobs = 1 << 16;

// pass 2: U and V of every block from its frozen pivots (same arithmetic as the
// search), written into the final layout; U and V are cleared first (padding)
void form_factors(Handle &h, cudaStream_t s, Arena &tmp, int64_t budget, const BlockGeometry &g,
                  const std::vector<int> &rk, const std::vector<int64_t> &poff_h) {
    const int64_t nblk = h.nblk;
    const size_t es = h.elem();
    H3D_CUDA(cudaMemsetAsync(h.U, 0, (size_t)std::max<int64_t>(h.u_elems, 4) * es, s));
    H3D_CUDA(cudaMemsetAsync(h.V, 0, (size_t)std::max<int64_t>(h.v_elems, 4) * es, s));
    size_t free_b = 0, total_b = 0;
    H3D_CUDA(cudaMemGetInfo(&free_b, &total_b));
    int64_t ws2 = budget > 0 ? budget : std::min<int64_t>((int64_t)(free_b * 0.6), (int64_t)48 << 30);
    int64_t dbl2 = std::max<int64_t>(ws2 / 8, (int64_t)8 << 20);
    int64_t maxneed = 0;
    for (int64_t b = 0; b < nblk; ++b) maxneed = std::max(maxneed, (int64_t)rk[b] * (g.m(b) + g.n(b)));
    dbl2 = std::max(dbl2, maxneed);
    double *scratch2 = (double *)tmp.alloc((size_t)dbl2 * 8);
    AcaJob *d_jobs = tmp.get<AcaJob>((size_t)kMaxJobs);
    AcaArgs A{};
    A.px = h.px; A.py = h.py; A.pz = h.pz;
    A.kind = h.kernel; A.kappa = h.kappa; A.tol = h.tol;
    A.rank = h.rank; A.err = h.d_err;
    A.scratch = scratch2; A.flags = nullptr; A.sig = h.sigma; A.tau = h.tau;
    const int64_t offL = h.box_off[h.L];
    PackArgs P{h.blk_tgt, h.blk_src, h.cu, h.cv, h.R, h.ldv, h.box_leaf_lo, h.leaf_ld, h.point_leaf, h.box_start,
               h.ubase, h.vbase, h.leaf_lp, offL};
    const bool sym = h.symmetric();
    if (sym) H3D_CUDA(cudaMemsetAsync(h.symF, 0, (size_t)std::max<int64_t>(h.sym_elems, 4) * es, s));
    // symmetric storage: pack jobs (pairs in the U / V layout, both orders) and fused pairs
    AcaJob *d_pack = sym ? tmp.get<AcaJob>((size_t)2 * kMaxJobs) : nullptr;
    std::vector<AcaJob> small, large, all, fused;
    int mcs = 0, mcl = 0;
    int64_t used = 0;
    auto pack = [&](const AcaJob *d, int cnt) {
        if (cnt == 0) return;
        if (h.prec == H3D_FP64)
            k_pack<double><<<(unsigned)cnt, kThreads, 0, s>>>(d, cnt, scratch2, P, (double *)h.U, (double *)h.V);
        else
            k_pack<float><<<(unsigned)cnt, kThreads, 0, s>>>(d, cnt, scratch2, P, (float *)h.U, (float *)h.V);
        H3D_LAUNCH_CHECK();
    };
    auto flush = [&]() {
        if (small.empty() && large.empty()) return;
        run_batch<true>(small, large, mcs, mcl, A, d_jobs, s);
        all.clear();
        all.insert(all.end(), small.begin(), small.end());
        all.insert(all.end(), large.begin(), large.end());
        if (!sym) {
            pack(d_jobs, (int)all.size());
        } else {
            // a pair in the U / V layout is packed for (X, Y) and, transposed, for
            // (Y, X): the mirror's U is the primary's V and the other way round
            std::vector<AcaJob> both;
            fused.clear();
            for (const AcaJob &J : all) {
                if (h.sym_slot_h[J.blk] >= 0) {
                    fused.push_back(J);
                    continue;
                }
                both.push_back(J);
                AcaJob M = J;
                M.blk = g.partner[J.blk];
                M.m = J.n; M.n = J.m; M.xs = J.ys; M.ys = J.xs;
                M.uoff = J.voff; M.voff = J.uoff;
                both.push_back(M);
            }
            if (!both.empty()) {
                H3D_CUDA(cudaMemcpyAsync(d_pack, both.data(), both.size() * sizeof(AcaJob), cudaMemcpyHostToDevice, s));
                pack(d_pack, (int)both.size());
            }
            if (!fused.empty()) {
                AcaJob *d_f = d_pack + both.size();
                H3D_CUDA(cudaMemcpyAsync(d_f, fused.data(), fused.size() * sizeof(AcaJob), cudaMemcpyHostToDevice, s));
                if (h.prec == H3D_FP64)
                    k_pack_sym<double><<<(unsigned)fused.size(), kThreads, 0, s>>>(
                        d_f, (int)fused.size(), scratch2, h.sym_slot, h.sym_blk, (double *)h.symF);
                else
                    k_pack_sym<float><<<(unsigned)fused.size(), kThreads, 0, s>>>(
                        d_f, (int)fused.size(), scratch2, h.sym_slot, h.sym_blk, (float *)h.symF);
                H3D_LAUNCH_CHECK();
            }
        }
        H3D_CUDA(cudaStreamSynchronize(s));
        small.clear(); large.clear();
        mcs = mcl = 0; used = 0;
    };
    for (int64_t b = 0; b < nblk; ++b) {
        const int r = rk[b];
        if (r == 0 || g.mirror(b)) continue;
        const int m = g.m(b), n = g.n(b);
        const int64_t need = (int64_t)r * (m + n);
        if (used + need > dbl2 || (int64_t)(small.size() + large.size()) >= kMaxJobs) flush();
        AcaJob J;
        J.blk = (int)b; J.m = m; J.n = n; J.cap = r;
        J.xs = g.bstart[g.tgt[b]]; J.ys = g.bstart[g.src[b]];
        J.uoff = used; J.voff = used + (int64_t)r * m; J.foff = 0;
        J.poff = poff_h[b];  // frozen pivots are read from the final arrays
        used += need;
        if (std::max(m, n) <= kSmallMax) { small.push_back(J); mcs = std::max(mcs, r); }
        else { large.push_back(J); mcl = std::max(mcl, r); }
    }
    flush();
    if (d_pack) tmp.free_one(d_pack);
    tmp.free_one(d_jobs);
    tmp.free_one(scratch2);
}

// Pivots given by the caller: checked (0 <= r <= min(m, n, rank_cap), indices
// inside the block, no index twice in one block) and uploaded.
void import_pivots(Handle &h, const FrozenPivots &fp, const BlockGeometry &g, std::vector<int> &rk,
                   std::vector<int64_t> &poff_h, cudaStream_t s) {
    const int64_t nblk = h.nblk;
    int maxdim = 1;
    for (int64_t b = 0; b < nblk; ++b) maxdim = std::max(maxdim, std::max(g.m(b), g.n(b)));
    std::vector<int64_t> seen_row((size_t)maxdim, -1), seen_col((size_t)maxdim, -1);
    for (int64_t b = 0; b < nblk; ++b) {
        const int r = fp.rank[b], m = g.m(b), n = g.n(b);
        if (r < 0 || r > std::min(std::min(m, n), h.rank_cap)) fail(H3D_ERR_ARG);
        rk[b] = r;
        poff_h[b + 1] = poff_h[b] + r;
        for (int64_t k = poff_h[b]; k < poff_h[b + 1]; ++k) {
            const int i = fp.sigma[k], j = fp.tau[k];
            if (i < 0 || i >= m || j < 0 || j >= n || seen_row[i] == b || seen_col[j] == b) fail(H3D_ERR_ARG);
            seen_row[i] = b;
            seen_col[j] = b;
        }
    }
    for (int64_t b = 0; b < nblk; ++b) {   // symmetric storage: mirrors carry the swapped pivots
        if (!g.mirror(b)) continue;
        const int p = g.partner[b];
        if (rk[b] != rk[p]) fail(H3D_ERR_ARG);
        for (int k = 0; k < rk[b]; ++k)
            if (fp.sigma[poff_h[b] + k] != fp.tau[poff_h[p] + k] || fp.tau[poff_h[b] + k] != fp.sigma[poff_h[p] + k])
                fail(H3D_ERR_ARG);
    }
    h.sum_rank = poff_h[nblk];
    if (nblk > 0) {
        H3D_CUDA(cudaMemcpyAsync(h.rank, rk.data(), nblk * sizeof(int), cudaMemcpyHostToDevice, s));
        H3D_CUDA(cudaMemcpyAsync(h.piv_off, poff_h.data(), (nblk + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    } else {
        H3D_CUDA(cudaMemcpyAsync(h.piv_off, poff_h.data(), sizeof(int64_t), cudaMemcpyHostToDevice, s));
    }
    h.sigma = h.mem.get<int>((size_t)std::max<int64_t>(h.sum_rank, 1));
    h.tau = h.mem.get<int>((size_t)std::max<int64_t>(h.sum_rank, 1));
    if (h.sum_rank > 0) {
        H3D_CUDA(cudaMemcpyAsync(h.sigma, fp.sigma, h.sum_rank * sizeof(int), cudaMemcpyHostToDevice, s));
        H3D_CUDA(cudaMemcpyAsync(h.tau, fp.tau, h.sum_rank * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    H3D_CUDA(cudaStreamSynchronize(s));
}

// Symmetric storage: the pairs whose factors fit one shared-memory stage (rank
// at most kSymMaxR), in list order, packed into groups that one bulk copy
// brings in: a pair that a warp can take (rank <= kSymSmallR, at most
// kSymSmallElems entries) joins the open group while the stage has room and the
// group has fewer than kSymGroupPairs pairs (one per warp); a larger one gets a
// group of its own.  Their ranks leave the U / V layout.  (A block of size el
// entries has el >= 2, so no small pair sorts with the key -1 of the large ones.)
void plan_symmetric(Handle &h, const BlockGeometry &g, const std::vector<int> &rk, std::vector<int> &lrk,
                    cudaStream_t s) {
    const int64_t nblk = h.nblk;
    const int64_t es = (int64_t)h.elem();
    const int64_t stage = es == 8 ? kSymStageF64 : kSymStageF32;
    std::vector<SymBlk> blks;
    std::vector<SymGroup> grps;
    h.sym_slot_h.assign((size_t)nblk, -1);
    h.sym_entries = 0;
    int64_t off = 0;
    SymGroup cur{};
    bool open = false;
    auto close = [&]() {
        if (!open) return;
        cur.bytes = (int)round_up((off - cur.off) * es, 16);
        off = cur.off + cur.bytes / es;
        grps.push_back(cur);
        open = false;
    };
    // the fused pairs: those a CTA takes in list order, then those a warp takes
    // from the largest down, so that the pairs of one group (one per warp, all
    // waited for together) are of about the same size
    std::vector<std::pair<int64_t, int64_t>> order;   // (sort key, block)
    for (int64_t b = 0; b < nblk; ++b) {
        if (g.mirror(b)) continue;
        const int r = rk[b];
        if (r == 0 || r > kSymMaxR) continue;
        const int m = g.m(b), n = g.n(b);
        const int64_t el = (int64_t)r * (sym_ld(m) + sym_ld(n));
        if (el * es > stage) continue;
        const bool big = r > kSymSmallR || el > kSymSmallElems;
        order.push_back({big ? -1 : -el, b});
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<int64_t, int64_t> &a, const std::pair<int64_t, int64_t> &c) {
                         return (a.first == -1) != (c.first == -1) ? a.first == -1 : a.first < c.first;
                     });
    for (const auto &ob : order) {
        const int64_t b = ob.second;
        const int r = rk[b];
        const int m = g.m(b), n = g.n(b), ldm = sym_ld(m), ldn = sym_ld(n);
        const int64_t el = (int64_t)r * (ldm + ldn);
        const bool big = ob.first == -1;
        if (big || !open || (off - cur.off + el) * es > stage || cur.nb >= kSymGroupPairs) {
            close();
            cur = SymGroup{};
            cur.off = off;
            cur.b0 = (int)blks.size();
            cur.big = big ? 1 : 0;
            open = true;
        }
        SymBlk B{};
        B.off = off;
        B.xs = g.bstart[g.tgt[b]]; B.ys = g.bstart[g.src[b]];
        B.m = m; B.n = n; B.r = r; B.ldm = ldm; B.ldn = ldn;
        h.sym_slot_h[b] = (int)blks.size();
        blks.push_back(B);
        off += el;
        ++cur.nb;
        if (big) close();
        lrk[b] = 0;
        lrk[g.partner[b]] = 0;
        h.sym_entries += (int64_t)r * (m + n);
    }
    close();
    h.nsym = (int)blks.size();
    h.nsym_grp = (int)grps.size();
    h.sym_elems = off;
    h.sym_blk = h.mem.get<SymBlk>(std::max<size_t>(blks.size(), 1));
    h.sym_grp = h.mem.get<SymGroup>(std::max<size_t>(grps.size(), 1));
    h.sym_slot = h.mem.get<int>((size_t)std::max<int64_t>(nblk, 1));
    if (!blks.empty())
        H3D_CUDA(cudaMemcpyAsync(h.sym_blk, blks.data(), blks.size() * sizeof(SymBlk), cudaMemcpyHostToDevice, s));
    if (!grps.empty())
        H3D_CUDA(cudaMemcpyAsync(h.sym_grp, grps.data(), grps.size() * sizeof(SymGroup), cudaMemcpyHostToDevice, s));
    if (nblk > 0)
        H3D_CUDA(cudaMemcpyAsync(h.sym_slot, h.sym_slot_h.data(), nblk * sizeof(int), cudaMemcpyHostToDevice, s));
    H3D_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

void build_factors(Handle &h, cudaStream_t s, Arena &tmp, int64_t budget, const FrozenPivots *fp) {
    const int64_t nblk = h.nblk, nboxes = h.n_boxes;
    const int vw = h.prec == H3D_FP64 ? 2 : 4;
    const int64_t offL = h.box_off[h.L];
    h.rank = h.mem.get<int>((size_t)std::max<int64_t>(nblk, 1));
    h.piv_off = h.mem.get<int64_t>((size_t)nblk + 1);
    H3D_CUDA(cudaMemsetAsync(h.rank, 0, sizeof(int) * (size_t)std::max<int64_t>(nblk, 1), s));

    const BlockGeometry g = block_geometry(h, s);
    std::vector<int> rk(nblk);
    std::vector<int64_t> poff_h(nblk + 1, 0);
    if (fp) {
        import_pivots(h, *fp, g, rk, poff_h, s);
    } else {
        size_t free_b = 0, total_b = 0;
        H3D_CUDA(cudaMemGetInfo(&free_b, &total_b));
        int64_t ws = budget > 0 ? budget : std::min<int64_t>((int64_t)(free_b * 0.45), (int64_t)48 << 30);
        ws = std::max<int64_t>(ws, (int64_t)64 << 20);

        AcaArgs A{};
        A.px = h.px; A.py = h.py; A.pz = h.pz;
        A.kind = h.kernel; A.kappa = h.kappa; A.tol = h.tol;
        A.rank = h.rank; A.err = h.d_err;

        // ---------------- pass 1: pivots and ranks
        int64_t piv_slots = 0;
        std::vector<int64_t> slot(nblk);
        for (int64_t b = 0; b < nblk; ++b) {
            slot[b] = piv_slots;
            piv_slots += std::min(std::min(g.m(b), g.n(b)), h.rank_cap);
        }
        int *ssig = tmp.get<int>((size_t)std::max<int64_t>(piv_slots, 1));
        int *stau = tmp.get<int>((size_t)std::max<int64_t>(piv_slots, 1));
        const int64_t flag_ws = std::max<int64_t>(ws / 16, (int64_t)16 << 20);
        const int64_t dbl_ws = (ws - flag_ws) / 8;
        double *scratch = (double *)tmp.alloc((size_t)dbl_ws * 8);
        unsigned char *flags = tmp.get<unsigned char>((size_t)flag_ws);
        A.scratch = scratch; A.flags = flags; A.sig = ssig; A.tau = stau;
        H3D_CUDA(cudaMemsetAsync(h.d_err, 0, sizeof(int), s));

        AcaJob *d_jobs = tmp.get<AcaJob>((size_t)kMaxJobs);
        {
            std::vector<AcaJob> small, large;
            int mcs = 0, mcl = 0;
            int64_t used = 0, fused = 0;
            auto flush = [&]() {
                if (small.empty() && large.empty()) return;
                run_batch<false>(small, large, mcs, mcl, A, d_jobs, s);
                H3D_CUDA(cudaStreamSynchronize(s));  // job arrays are reused
                small.clear(); large.clear();
                mcs = mcl = 0; used = fused = 0;
            };
            for (int64_t b = 0; b < nblk; ++b) {
                if (g.mirror(b)) continue;   // symmetric storage: compressed as its primary
                const int m = g.m(b), n = g.n(b);
                const int cap = std::min(std::min(m, n), h.rank_cap);
                const int64_t need = (int64_t)cap * (m + n);
                if (need > dbl_ws || (int64_t)(m + n) > flag_ws) fail(H3D_ERR_OOM);
                if (used + need > dbl_ws || fused + m + n > flag_ws ||
                    (int64_t)(small.size() + large.size()) >= kMaxJobs)
                    flush();
                AcaJob J;
                J.blk = (int)b; J.m = m; J.n = n; J.cap = cap;
                J.xs = g.bstart[g.tgt[b]]; J.ys = g.bstart[g.src[b]];
                J.uoff = used; J.voff = used + (int64_t)cap * m; J.foff = fused; J.poff = slot[b];
                used += need; fused += m + n;
                if (std::max(m, n) <= kSmallMax) { small.push_back(J); mcs = std::max(mcs, cap); }
                else { large.push_back(J); mcl = std::max(mcl, cap); }
            }
            flush();
        }
        if (read_scalar(h.d_err, s) & (1 << H3D_ERR_ACA_RANK)) fail(H3D_ERR_ACA_RANK);

        // ranks -> pivot offsets, compact pivots (a mirror takes its primary's rank)
        if (nblk > 0) {
            H3D_CUDA(cudaMemcpyAsync(rk.data(), h.rank, nblk * sizeof(int), cudaMemcpyDeviceToHost, s));
            H3D_CUDA(cudaStreamSynchronize(s));
        }
        if (!g.partner.empty()) {
            for (int64_t b = 0; b < nblk; ++b)
                if (g.mirror(b)) rk[b] = rk[g.partner[b]];
            if (nblk > 0) H3D_CUDA(cudaMemcpyAsync(h.rank, rk.data(), nblk * sizeof(int), cudaMemcpyHostToDevice, s));
        }
        h.sum_rank = scan_exclusive(h.rank, h.piv_off, nblk, s, tmp);
        H3D_CUDA(cudaMemcpyAsync(h.piv_off + nblk, &h.sum_rank, sizeof(int64_t), cudaMemcpyHostToDevice, s));
        H3D_CUDA(cudaStreamSynchronize(s));
        for (int64_t b = 0; b < nblk; ++b) poff_h[b + 1] = poff_h[b] + rk[b];
        h.sigma = h.mem.get<int>((size_t)std::max<int64_t>(h.sum_rank, 1));
        h.tau = h.mem.get<int>((size_t)std::max<int64_t>(h.sum_rank, 1));
        for (int64_t b0 = 0; b0 < nblk; b0 += kMaxJobs) {
            const int64_t nb = std::min(kMaxJobs, nblk - b0);
            // own pivots first; then the mirrors, whose rows are their primary's
            // columns (the pivot arrays passed the other way round)
            std::vector<AcaJob> jobs, mir;
            for (int64_t q = 0; q < nb; ++q) {
                AcaJob J{};
                J.blk = (int)(b0 + q);
                if (g.mirror(b0 + q)) {
                    J.poff = slot[g.partner[b0 + q]];
                    mir.push_back(J);
                } else {
                    J.poff = slot[b0 + q];
                    jobs.push_back(J);
                }
            }
            const size_t nj = jobs.size();
            jobs.insert(jobs.end(), mir.begin(), mir.end());
            H3D_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(AcaJob), cudaMemcpyHostToDevice, s));
            if (nj > 0)
                k_copy_pivots<<<(unsigned)nj, 64, 0, s>>>(d_jobs, (int)nj, h.rank, h.piv_off, ssig, stau, h.sigma, h.tau);
            if (!mir.empty())
                k_copy_pivots<<<(unsigned)mir.size(), 64, 0, s>>>(d_jobs + nj, (int)mir.size(), h.rank, h.piv_off, stau,
                                                                  ssig, h.sigma, h.tau);
            H3D_LAUNCH_CHECK();
            H3D_CUDA(cudaStreamSynchronize(s));
        }
        tmp.free_one(ssig);
        tmp.free_one(stau);
        tmp.free_one(d_jobs);
        tmp.free_one(scratch);
        tmp.free_one(flags);
    }
    h.max_rank = 0;
    for (int64_t b = 0; b < nblk; ++b) h.max_rank = std::max(h.max_rank, rk[b]);

    // ---------------- symmetric storage: the fused pairs and the layout ranks
    std::vector<int> lrk;
    if (h.symmetric()) {
        lrk = rk;
        sym_prepare();
        plan_symmetric(h, g, rk, lrk, s);
        h.lrank = h.mem.get<int>((size_t)std::max<int64_t>(nblk, 1));
        if (nblk > 0) H3D_CUDA(cudaMemcpyAsync(h.lrank, lrk.data(), nblk * sizeof(int), cudaMemcpyHostToDevice, s));
    } else {
        h.lrank = h.rank;
    }
    const std::vector<int> &lr = h.symmetric() ? lrk : rk;

    // ---------------- layout
    h.R = h.mem.get<int>((size_t)nboxes);
    h.cu = h.mem.get<int>((size_t)std::max<int64_t>(nblk, 1));
    h.Rv = h.mem.get<int>((size_t)nboxes);
    h.ldv = h.mem.get<int>((size_t)nboxes);
    h.cv = h.mem.get<int>((size_t)std::max<int64_t>(nblk, 1));
    k_target_cols<<<gridn(nboxes), kThreads, 0, s>>>(h.tgt_ptr, h.lrank, nboxes, h.R, h.cu);
    H3D_LAUNCH_CHECK();
    H3D_CUDA(cudaMemsetAsync(h.d_err, 0, sizeof(int), s));
    k_source_cols<<<gridn(nboxes), kThreads, 0, s>>>(h.tgt_ptr, h.blk_partner, h.lrank, nboxes, vw, h.Rv, h.ldv, h.cv,
                                                      h.d_err);
    H3D_LAUNCH_CHECK();
    if (read_scalar(h.d_err, s) & (1 << H3D_ERR_STATE)) fail(H3D_ERR_STATE);
    h.tofs = h.mem.get<int64_t>((size_t)std::max<int64_t>(nblk, 1));
    scan_exclusive(h.lrank, h.tofs, nblk, s, tmp);
    h.tbase = h.mem.get<int64_t>((size_t)nboxes);
    scan_exclusive(h.R, h.tbase, nboxes, s, tmp);
    h.vcol0 = h.mem.get<int64_t>((size_t)nboxes);
    scan_exclusive(h.Rv, h.vcol0, nboxes, s, tmp);
    h.leaf_ld = h.mem.get<int>((size_t)h.nleaf + 1);
    H3D_CUDA(cudaMemsetAsync(h.leaf_ld, 0, sizeof(int) * ((size_t)h.nleaf + 1), s));
    k_leaf_ld<<<gridn(h.nleaf), kThreads, 0, s>>>(h.box_start, h.box_end, offL, h.nleaf, vw, h.leaf_ld);
    H3D_LAUNCH_CHECK();
    h.leaf_lp = h.mem.get<int64_t>((size_t)h.nleaf + 1);
    scan_exclusive(h.leaf_ld, h.leaf_lp, h.nleaf + 1, s, tmp);
    int64_t *usz = tmp.get<int64_t>((size_t)nboxes), *vsz = tmp.get<int64_t>((size_t)nboxes);
    k_box_sizes<<<gridn(nboxes), kThreads, 0, s>>>(h.box_start, h.box_end, h.R, h.ldv, h.box_leaf_lo, h.box_leaf_hi,
                                                    h.leaf_lp, nboxes, usz, vsz);
    H3D_LAUNCH_CHECK();
    h.ubase = h.mem.get<int64_t>((size_t)nboxes);
    h.vbase = h.mem.get<int64_t>((size_t)nboxes);
    h.u_elems = scan_exclusive(usz, h.ubase, nboxes, s, tmp);
    h.v_elems = scan_exclusive(vsz, h.vbase, nboxes, s, tmp);
    tmp.free_one(usz);
    tmp.free_one(vsz);
    h.map_v = h.mem.get<int64_t>((size_t)std::max<int64_t>(h.sum_rank, 1));
    if (nblk > 0) {
        k_map_v<<<gridn(nblk), kThreads, 0, s>>>(h.blk_src, h.lrank, h.cv, h.vcol0, h.tofs, nblk, h.map_v);
        H3D_LAUNCH_CHECK();
    }
    // entries stored (symmetric storage: the layout's pairs in both orders, the
    // fused pairs once)
    h.u_entries = h.v_entries = 0;
    for (int64_t b = 0; b < nblk; ++b) {
        const int r = lr[b] > 0 ? lr[b] : (h.symmetric() && h.sym_slot_h[b] >= 0 ? rk[b] : 0);
        h.u_entries += (int64_t)r * g.m(b);
        h.v_entries += (int64_t)r * g.n(b);
    }
    h.factor_entries = h.u_entries + h.v_entries;

    if (h.storage == H3D_STORE_SKELETON) {   // pivots and K(sigma,tau) only: no U, V
        build_skeleton(h, s, tmp);
        return;
    }
    const size_t es = h.elem();
    h.U = h.mem.alloc((size_t)std::max<int64_t>(h.u_elems, 4) * es);
    h.V = h.mem.alloc((size_t)std::max<int64_t>(h.v_elems, 4) * es);
    if (h.symmetric()) {
        h.symF = h.mem.alloc((size_t)std::max<int64_t>(h.sym_elems, 4) * es);
        h.sym_acc = h.mem.get<double>((size_t)h.N * 8);
    }

    // ---------------- pass 2: frozen pivots -> U, V -> final layout
    form_factors(h, s, tmp, budget, g, rk, poff_h);
}

void reform_factors(Handle &h, cudaStream_t s, Arena &tmp) {
    const int64_t nblk = h.nblk;
    const BlockGeometry g = block_geometry(h, s);
    std::vector<int> rk(nblk);
    std::vector<int64_t> poff_h(nblk + 1, 0);
    if (nblk > 0) {
        H3D_CUDA(cudaMemcpyAsync(rk.data(), h.rank, nblk * sizeof(int), cudaMemcpyDeviceToHost, s));
        H3D_CUDA(cudaStreamSynchronize(s));
    }
    for (int64_t b = 0; b < nblk; ++b) poff_h[b + 1] = poff_h[b] + rk[b];
    form_factors(h, s, tmp, h.budget, g, rk, poff_h);
}

}  // namespace h3d
