// h3d_tree.cu -- octree (Sec. 2.1), neighbour classes and interaction lists
// (Table "Notations", Definition admh3d, Alg. 1 first two steps), on the GPU.
//
//   A1  Morton key per point: 21 bits per axis, x the most significant bit of
//       each triple; cell index floor(((x - lo) / side) * 2^21), clamped.
//   A2  stable radix sort of (key, index); depth L = the first level at which
//       no box holds more than leaf_size points; boxes per level by boundary
//       flags and a prefix sum.
//   A3  for every box, candidates are the children of the parent's self, face
//       and edge neighbours (the clan); vertex-sharing and well-separated
//       candidates form the interaction list.  At the leaf level the self,
//       face and edge neighbours form the dense near list.
#include <algorithm>

#include "h3d_internal.cuh"

namespace h3d {

namespace {

constexpr int kT = 256;

inline unsigned grid_for(int64_t n, int t = kT) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

__device__ __forceinline__ uint64_t spread_bits3(uint64_t v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__global__ void k_morton(const double *__restrict__ pts, int64_t n, double lo0, double lo1, double lo2,
                         double side, uint64_t *__restrict__ keys, int *__restrict__ idx, int *__restrict__ err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double lo[3] = {lo0, lo1, lo2};
    uint64_t c[3];
    bool bad = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double t = __ddiv_rn(__dsub_rn(pts[3 * i + d], lo[d]), side);
        if (!(t >= 0.0 && t <= 1.0)) {
            bad = true;
            t = 0.0;
        }
        double u = floor(__dmul_rn(t, 2097152.0));
        uint64_t q = (uint64_t)u;
        c[d] = q > 2097151ull ? 2097151ull : q;
    }
    if (bad) atomicOr(err, 1 << H3D_ERR_DOMAIN);
    keys[i] = (spread_bits3(c[0]) << 2) | (spread_bits3(c[1]) << 1) | spread_bits3(c[2]);
    idx[i] = (int)i;
}

// number of octree levels (0..21) on which two keys fall in the same box
__device__ __forceinline__ int shared_levels(uint64_t a, uint64_t b) {
    uint64_t x = a ^ b;
    int c = __clzll((long long)x);  // top bit of a 63-bit key is always 0
    int s = (c - 1) / 3;
    return s > kMaxDepth ? kMaxDepth : s;
}

__global__ void k_depth(const uint64_t *__restrict__ keys, int64_t n, int leaf, int *__restrict__ maxshared) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int s = -1;
    if (i + leaf < n) s = shared_levels(keys[i], keys[i + leaf]);
    // warp max then one atomic
    for (int o = 16; o > 0; o >>= 1) s = max(s, __shfl_xor_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0 && s >= 0) atomicMax(maxshared, s);
}

// first level at which point i opens a new box (22 = never)
__global__ void k_first_level(const uint64_t *__restrict__ keys, int64_t n, unsigned char *__restrict__ fl,
                              int *__restrict__ hist) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int f = 0;
    if (i > 0) {
        uint64_t x = keys[i] ^ keys[i - 1];
        f = x == 0 ? kMaxDepth + 1 : ((__clzll((long long)x) - 1) / 3) + 1;
        if (f > kMaxDepth + 1) f = kMaxDepth + 1;
    }
    fl[i] = (unsigned char)f;
    atomicAdd(&hist[f], 1);
}

__global__ void k_flags(const unsigned char *__restrict__ fl, int64_t n, int level, int *__restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = fl[i] <= level ? 1 : 0;
}

__global__ void k_level_fill(const uint64_t *__restrict__ keys, const int *__restrict__ flag,
                             const int64_t *__restrict__ pos, int64_t n, int shift, int64_t off,
                             uint64_t *__restrict__ box_key, int *__restrict__ box_start,
                             int *__restrict__ point_box) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = pos[i] + flag[i] - 1;
    point_box[i] = (int)(off + b);
    if (flag[i]) {
        box_key[off + b] = keys[i] >> shift;
        box_start[off + b] = (int)i;
    }
}

__global__ void k_level_ends(const int *__restrict__ box_start, int *__restrict__ box_end, int64_t off, int nb,
                             int64_t n) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    box_end[off + b] = b + 1 < nb ? box_start[off + b + 1] : (int)n;
}

__global__ void k_parents(const int *__restrict__ box_start, const int *__restrict__ point_box_prev,
                          int *__restrict__ parent, int64_t off, int nb) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    parent[off + b] = point_box_prev[box_start[off + b]];
}

__global__ void k_gather_points(const double *__restrict__ pts, const int *__restrict__ perm, int64_t n,
                                double *__restrict__ px, double *__restrict__ py, double *__restrict__ pz) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = perm[i];
    px[i] = pts[3 * o];
    py[i] = pts[3 * o + 1];
    pz[i] = pts[3 * o + 2];
}

__global__ void k_leaf_info(const int *__restrict__ box_start, const int *__restrict__ box_end,
                            const int *__restrict__ point_leaf_global, int64_t off_leaf, int64_t nboxes,
                            int *__restrict__ leaf_lo, int *__restrict__ leaf_hi) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nboxes) return;
    leaf_lo[g] = (int)(point_leaf_global[box_start[g]] - off_leaf);
    leaf_hi[g] = (int)(point_leaf_global[box_end[g] - 1] - off_leaf) + 1;
}

__global__ void k_point_leaf(const int *__restrict__ point_leaf_global, int64_t n, int64_t off_leaf,
                             int *__restrict__ point_leaf) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) point_leaf[i] = (int)(point_leaf_global[i] - off_leaf);
}

__global__ void k_ancestors(const int *__restrict__ parent, int64_t off_leaf, int nleaf, int L,
                            int *__restrict__ anc) {
    int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= nleaf) return;
    int a = (int)(off_leaf + z);
    for (int l = L; l >= 1; --l) {
        anc[(int64_t)(l - 1) * nleaf + z] = a;
        a = parent[a];
    }
}

__global__ void k_local_coords(const double *__restrict__ px, const double *__restrict__ py,
                               const double *__restrict__ pz, const int *__restrict__ point_leaf,
                               const uint64_t *__restrict__ box_key, int64_t off_leaf, int L, double lo0,
                               double lo1, double lo2, double h, int64_t n, float4 *__restrict__ ploc,
                               float4 *__restrict__ ploc_lo) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int x, y, z;
    box_coords(box_key[off_leaf + point_leaf[i]], L, x, y, z);
    const double cx = lo0 + (x + 0.5) * h, cy = lo1 + (y + 0.5) * h, cz = lo2 + (z + 0.5) * h;
    const double dx = px[i] - cx, dy = py[i] - cy, dz = pz[i] - cz;
    const float hx = (float)dx, hy = (float)dy, hz = (float)dz;
    ploc[i] = make_float4(hx, hy, hz, 0.0f);
    ploc_lo[i] = make_float4((float)(dx - (double)hx), (float)(dy - (double)hy), (float)(dz - (double)hz), 0.0f);
}

// new coordinates for the sorted points: flags[0] |= 1 if any differs from the
// current ones, flags[0] |= 2 if any is not finite
__global__ void k_points_differ(const double *__restrict__ pts, const int *__restrict__ perm, int64_t n,
                                const double *__restrict__ px, const double *__restrict__ py,
                                const double *__restrict__ pz, int *__restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = perm[i];
    const double x = pts[3 * o], y = pts[3 * o + 1], z = pts[3 * o + 2];
    int f = 0;
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) f |= 2;
    // bit patterns, so that -0.0 and 0.0 count as different and NaN is caught above
    if (__double_as_longlong(x) != __double_as_longlong(px[i]) ||
        __double_as_longlong(y) != __double_as_longlong(py[i]) ||
        __double_as_longlong(z) != __double_as_longlong(pz[i]))
        f |= 1;
    if (f) atomicOr(flags, f);
}

__global__ void k_scatter_points(const double *__restrict__ px, const double *__restrict__ py,
                                 const double *__restrict__ pz, const int *__restrict__ perm, int64_t n,
                                 double *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = perm[i];
    out[3 * o] = px[i];
    out[3 * o + 1] = py[i];
    out[3 * o + 2] = pz[i];
}

// ---------------------------------------------------------------------------
// lists

__device__ int find_box(const uint64_t *__restrict__ keys, int nb, uint64_t key) {
    int lo = 0, hi = nb;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    return (lo < nb && keys[lo] == key) ? lo : -1;
}

__device__ __forceinline__ int pair_class(int dx, int dy, int dz) {
    dx = abs(dx); dy = abs(dy); dz = abs(dz);
    if (max(dx, max(dy, dz)) >= 2) return 4;
    return (dx != 0) + (dy != 0) + (dz != 0);
}

// Admissibility of two distinct same-level boxes of class cls (0 self, 1 face,
// 2 edge, 3 vertex, 4 well separated):
//   HODLR3D (Def. admh3d): vertex or well separated;
//   strong, eta = sqrt(3) (Eq. adm): well separated only;
//   weak (HODLR on the octree): every distinct pair.
__device__ __forceinline__ bool is_admissible(int cls, int mode) {
    if (mode == H3D_ADM_STRONG) return cls == 4;
    if (mode == H3D_ADM_WEAK) return cls != 0;
    return cls == 3 || cls == 4;
}

// Interaction list of box i at level l (l >= 1): the children of the parent's
// neighbours whose pair with the parent was not admissible (for HODLR3D the
// clan: siblings and children of the parent's edge / face neighbours) that are
// admissible themselves.  Writes up to 215 sorted level-local indices with their
// class; returns the count.
constexpr int kMaxIList = 216;
__device__ int interaction_list(const uint64_t *__restrict__ bkey, int nb, int level, int i, int mode, int *out,
                                unsigned char *cls_out) {
    int x, y, z;
    box_coords(bkey[i], level, x, y, z);
    const int px = x >> 1, py = y >> 1, pz = z >> 1;
    const int np = 1 << (level - 1);
    int cnt = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                const int pcls = (dx != 0) + (dy != 0) + (dz != 0);
                if (pcls != 0 && is_admissible(pcls, mode)) continue;  // covered at the parent level
                const int qx = px + dx, qy = py + dy, qz = pz + dz;
                if (qx < 0 || qy < 0 || qz < 0 || qx >= np || qy >= np || qz >= np) continue;
                for (int c = 0; c < 8; ++c) {
                    const int cx = 2 * qx + ((c >> 2) & 1), cy = 2 * qy + ((c >> 1) & 1), cz = 2 * qz + (c & 1);
                    const int cls = pair_class(cx - x, cy - y, cz - z);
                    if (cls == 0 || !is_admissible(cls, mode)) continue;
                    const int j = find_box(bkey, nb, box_key_of(cx, cy, cz, level));
                    if (j < 0) continue;
                    if (out) {
                        // insertion into the sorted prefix
                        int p = cnt;
                        while (p > 0 && out[p - 1] > j) {
                            out[p] = out[p - 1];
                            cls_out[p] = cls_out[p - 1];
                            --p;
                        }
                        out[p] = j;
                        cls_out[p] = (unsigned char)cls;
                    }
                    ++cnt;
                }
            }
    return cnt;
}

__global__ void k_ilist_count(const uint64_t *__restrict__ bkey, int nb, int level, int mode, int *__restrict__ cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    cnt[i] = interaction_list(bkey, nb, level, i, mode, nullptr, nullptr);
}

__global__ void k_ilist_fill(const uint64_t *__restrict__ bkey, int nb, int level, int mode, int64_t off_box,
                             const int64_t *__restrict__ bptr, int *__restrict__ tgt, int *__restrict__ src,
                             unsigned char *__restrict__ cls, unsigned char *__restrict__ lev) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int js[kMaxIList];
    unsigned char cs[kMaxIList];
    const int n = interaction_list(bkey, nb, level, i, mode, js, cs);
    const int64_t o = bptr[off_box + i];
    for (int k = 0; k < n; ++k) {
        tgt[o + k] = (int)(off_box + i);
        src[o + k] = (int)(off_box + js[k]);
        cls[o + k] = cs[k];
        lev[o + k] = (unsigned char)level;
    }
}

// Near list of leaf i: itself and the neighbours whose pair is not admissible
// (HODLR3D: self, face and edge neighbours), sorted.
__device__ int near_list(const uint64_t *__restrict__ bkey, int nb, int level, int i, int mode, int *out,
                         unsigned char *cls_out, unsigned char *dir_out) {
    int x, y, z;
    box_coords(bkey[i], level, x, y, z);
    const int n1 = 1 << level;
    int cnt = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                const int cls = (dx != 0) + (dy != 0) + (dz != 0);
                if (cls != 0 && is_admissible(cls, mode)) continue;
                const int cx = x + dx, cy = y + dy, cz = z + dz;
                if (cx < 0 || cy < 0 || cz < 0 || cx >= n1 || cy >= n1 || cz >= n1) continue;
                const int j = find_box(bkey, nb, box_key_of(cx, cy, cz, level));
                if (j < 0) continue;
                if (out) {
                    int p = cnt;
                    while (p > 0 && out[p - 1] > j) {
                        out[p] = out[p - 1];
                        cls_out[p] = cls_out[p - 1];
                        dir_out[p] = dir_out[p - 1];
                        --p;
                    }
                    out[p] = j;
                    cls_out[p] = (unsigned char)cls;
                    dir_out[p] = (unsigned char)((dx + 1) * 9 + (dy + 1) * 3 + (dz + 1));
                }
                ++cnt;
            }
    return cnt;
}

__global__ void k_near_count(const uint64_t *__restrict__ bkey, int nb, int level, int mode, int *__restrict__ cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    cnt[i] = near_list(bkey, nb, level, i, mode, nullptr, nullptr, nullptr);
}

__global__ void k_near_fill(const uint64_t *__restrict__ bkey, int nb, int level, int mode,
                            const int64_t *__restrict__ nptr, int *__restrict__ src, unsigned char *__restrict__ cls,
                            unsigned char *__restrict__ dir) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int js[27];
    unsigned char cs[27], ds[27];
    const int n = near_list(bkey, nb, level, i, mode, js, cs, ds);
    const int64_t o = nptr[i];
    for (int k = 0; k < n; ++k) {
        src[o + k] = js[k];
        cls[o + k] = cs[k];
        dir[o + k] = ds[k];
    }
}

__global__ void k_i64_to_i32(const int64_t *__restrict__ in, int *__restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int)in[i];
}

__global__ void k_partner(const int *__restrict__ tgt, const int *__restrict__ src,
                          const int64_t *__restrict__ tptr, int64_t nblk, int *__restrict__ partner) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    const int X = tgt[b], Y = src[b];
    int64_t lo = tptr[Y], hi = tptr[Y + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (src[mid] < X) lo = mid + 1; else hi = mid;
    }
    partner[b] = (lo < tptr[Y + 1] && src[lo] == X) ? (int)lo : -1;
}

__global__ void k_near_sizes(const int *__restrict__ nptr, const int *__restrict__ nsrc,
                             const int *__restrict__ box_start, const int *__restrict__ box_end, int64_t off_leaf,
                             int nleaf, int64_t *__restrict__ out) {
    int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= nleaf) return;
    const int64_t m = box_end[off_leaf + z] - box_start[off_leaf + z];
    int64_t s = 0;
    for (int p = nptr[z]; p < nptr[z + 1]; ++p) {
        const int y = nsrc[p];
        s += m * (int64_t)(box_end[off_leaf + y] - box_start[off_leaf + y]);
    }
    out[z] = s;
}

}  // namespace

void build_tree(Handle &h, const double *points, cudaStream_t s, Arena &tmp) {
    const int64_t n = h.N;
    uint64_t *keys = h.mem.get<uint64_t>((size_t)n);
    int *idx = h.mem.get<int>((size_t)n);
    H3D_CUDA(cudaMemsetAsync(h.d_err, 0, sizeof(int), s));
    k_morton<<<grid_for(n), kT, 0, s>>>(points, n, h.lo[0], h.lo[1], h.lo[2], h.side, keys, idx, h.d_err);
    H3D_LAUNCH_CHECK();
    if (read_scalar(h.d_err, s) & (1 << H3D_ERR_DOMAIN)) fail(H3D_ERR_DOMAIN);
    radix_sort_pairs(keys, idx, n, 63, s, tmp);
    h.keys = keys;
    h.perm = idx;

    // depth
    int *d_ms = tmp.get<int>(1);
    H3D_CUDA(cudaMemsetAsync(d_ms, 0xff, sizeof(int), s));  // -1
    if (n > h.leaf_size) {
        k_depth<<<grid_for(n), kT, 0, s>>>(keys, n, h.leaf_size, d_ms);
        H3D_LAUNCH_CHECK();
    }
    const int ms = read_scalar(d_ms, s);
    h.L = ms < 0 ? 0 : ms + 1;
    if (h.L > kMaxDepth) fail(H3D_ERR_DEPTH);
    const int L = h.L;

    h.px = h.mem.get<double>((size_t)n);
    h.py = h.mem.get<double>((size_t)n);
    h.pz = h.mem.get<double>((size_t)n);
    k_gather_points<<<grid_for(n), kT, 0, s>>>(points, idx, n, h.px, h.py, h.pz);
    H3D_LAUNCH_CHECK();

    // boxes of every level
    unsigned char *fl = tmp.get<unsigned char>((size_t)n);
    int *hist = tmp.get<int>(kMaxDepth + 2);
    H3D_CUDA(cudaMemsetAsync(hist, 0, (kMaxDepth + 2) * sizeof(int), s));
    k_first_level<<<grid_for(n), kT, 0, s>>>(keys, n, fl, hist);
    H3D_LAUNCH_CHECK();
    int hh[kMaxDepth + 2];
    H3D_CUDA(cudaMemcpyAsync(hh, hist, sizeof(hh), cudaMemcpyDeviceToHost, s));
    H3D_CUDA(cudaStreamSynchronize(s));
    int64_t acc = 0, tot = 0;
    for (int l = 0; l <= L; ++l) {
        acc += hh[l];
        h.nbox[l] = (int)acc;
        h.box_off[l] = tot;
        tot += acc;
    }
    h.box_off[L + 1] = tot;
    h.n_boxes = tot;
    h.nleaf = h.nbox[L];
    h.box_key = h.mem.get<uint64_t>((size_t)tot);
    h.box_start = h.mem.get<int>((size_t)tot);
    h.box_end = h.mem.get<int>((size_t)tot);
    h.box_parent = h.mem.get<int>((size_t)tot);
    int *flag = tmp.get<int>((size_t)n);
    int64_t *pos = tmp.get<int64_t>((size_t)n);
    int *pb_prev = tmp.get<int>((size_t)n);
    int *pb_cur = tmp.get<int>((size_t)n);
    H3D_CUDA(cudaMemsetAsync(h.box_parent, 0xff, sizeof(int), s));  // root has no parent
    for (int l = 0; l <= L; ++l) {
        const int64_t off = h.box_off[l];
        const int nb = h.nbox[l];
        k_flags<<<grid_for(n), kT, 0, s>>>(fl, n, l, flag);
        H3D_LAUNCH_CHECK();
        scan_exclusive(flag, pos, n, s, tmp);
        k_level_fill<<<grid_for(n), kT, 0, s>>>(keys, flag, pos, n, 3 * (kMaxDepth - l), off, h.box_key,
                                                 h.box_start, pb_cur);
        H3D_LAUNCH_CHECK();
        k_level_ends<<<grid_for(nb), kT, 0, s>>>(h.box_start, h.box_end, off, nb, n);
        H3D_LAUNCH_CHECK();
        if (l > 0) {
            k_parents<<<grid_for(nb), kT, 0, s>>>(h.box_start, pb_prev, h.box_parent, off, nb);
            H3D_LAUNCH_CHECK();
        }
        std::swap(pb_prev, pb_cur);
    }
    // pb_prev now maps points to leaves (global index)
    const int64_t offL = h.box_off[L];
    h.point_leaf = h.mem.get<int>((size_t)n);
    k_point_leaf<<<grid_for(n), kT, 0, s>>>(pb_prev, n, offL, h.point_leaf);
    H3D_LAUNCH_CHECK();
    h.box_leaf_lo = h.mem.get<int>((size_t)tot);
    h.box_leaf_hi = h.mem.get<int>((size_t)tot);
    k_leaf_info<<<grid_for(tot), kT, 0, s>>>(h.box_start, h.box_end, pb_prev, offL, tot, h.box_leaf_lo,
                                               h.box_leaf_hi);
    H3D_LAUNCH_CHECK();
    h.leaf_anc = h.mem.get<int>((size_t)std::max(1, L) * h.nleaf);
    if (L > 0) {
        k_ancestors<<<grid_for(h.nleaf), kT, 0, s>>>(h.box_parent, offL, h.nleaf, L, h.leaf_anc);
        H3D_LAUNCH_CHECK();
    }
    h.ploc = h.mem.get<float4>((size_t)n);
    h.ploc_lo = h.mem.get<float4>((size_t)n);
    const double hL = h.side / (double)(1 << L);
    k_local_coords<<<grid_for(n), kT, 0, s>>>(h.px, h.py, h.pz, h.point_leaf, h.box_key, offL, L, h.lo[0],
                                                h.lo[1], h.lo[2], hL, n, h.ploc, h.ploc_lo);
    H3D_LAUNCH_CHECK();
}

void build_lists(Handle &h, cudaStream_t s, Arena &tmp) {
    const int L = h.L;
    const int64_t nboxes = h.n_boxes;
    // interaction lists: counts per global box, one scan gives the block offsets
    int *cnt = tmp.get<int>((size_t)nboxes + 1);
    H3D_CUDA(cudaMemsetAsync(cnt, 0, ((size_t)nboxes + 1) * sizeof(int), s));
    for (int l = 1; l <= L; ++l) {
        k_ilist_count<<<grid_for(h.nbox[l]), kT, 0, s>>>(h.box_key + h.box_off[l], h.nbox[l], l, h.adm,
                                                          cnt + h.box_off[l]);
        H3D_LAUNCH_CHECK();
    }
    h.tgt_ptr = h.mem.get<int64_t>((size_t)nboxes + 1);
    h.nblk = scan_exclusive(cnt, h.tgt_ptr, nboxes + 1, s, tmp);
    // blocks of level l start at the first box of level l
    for (int l = 0; l <= L + 1; ++l) {
        if (l <= L) h.blk_off[l] = read_scalar(h.tgt_ptr + h.box_off[l], s);
        else h.blk_off[l] = h.nblk;
    }
    const int64_t nblk = h.nblk;
    h.blk_tgt = h.mem.get<int>((size_t)std::max<int64_t>(nblk, 1));
    h.blk_src = h.mem.get<int>((size_t)std::max<int64_t>(nblk, 1));
    h.blk_cls = h.mem.get<unsigned char>((size_t)std::max<int64_t>(nblk, 1));
    h.blk_lev = h.mem.get<unsigned char>((size_t)std::max<int64_t>(nblk, 1));
    h.blk_partner = h.mem.get<int>((size_t)std::max<int64_t>(nblk, 1));
    for (int l = 1; l <= L; ++l) {
        k_ilist_fill<<<grid_for(h.nbox[l], 128), 128, 0, s>>>(h.box_key + h.box_off[l], h.nbox[l], l, h.adm,
                                                              h.box_off[l],
                                                              h.tgt_ptr, h.blk_tgt, h.blk_src, h.blk_cls, h.blk_lev);
        H3D_LAUNCH_CHECK();
    }
    if (nblk > 0) {
        k_partner<<<grid_for(nblk), kT, 0, s>>>(h.blk_tgt, h.blk_src, h.tgt_ptr, nblk, h.blk_partner);
        H3D_LAUNCH_CHECK();
    }
    // near lists at the leaf level
    const int nleaf = h.nleaf;
    const int64_t offL = h.box_off[L];
    int *ncnt = tmp.get<int>((size_t)nleaf + 1);
    H3D_CUDA(cudaMemsetAsync(ncnt, 0, ((size_t)nleaf + 1) * sizeof(int), s));
    k_near_count<<<grid_for(nleaf), kT, 0, s>>>(h.box_key + offL, nleaf, L, h.adm, ncnt);
    H3D_LAUNCH_CHECK();
    int64_t *nptr64 = tmp.get<int64_t>((size_t)nleaf + 1);
    h.nnear = scan_exclusive(ncnt, nptr64, nleaf + 1, s, tmp);
    h.near_ptr = h.mem.get<int>((size_t)nleaf + 1);
    k_i64_to_i32<<<grid_for(nleaf + 1), kT, 0, s>>>(nptr64, h.near_ptr, nleaf + 1);
    H3D_LAUNCH_CHECK();
    h.near_src = h.mem.get<int>((size_t)h.nnear);
    h.near_cls = h.mem.get<unsigned char>((size_t)h.nnear);
    h.near_dir = h.mem.get<unsigned char>((size_t)h.nnear);
    k_near_fill<<<grid_for(nleaf), kT, 0, s>>>(h.box_key + offL, nleaf, L, h.adm, nptr64, h.near_src, h.near_cls,
                                                 h.near_dir);
    H3D_LAUNCH_CHECK();
    int64_t *nsz = tmp.get<int64_t>((size_t)nleaf + 1);
    int64_t *nszp = tmp.get<int64_t>((size_t)nleaf + 1);
    H3D_CUDA(cudaMemsetAsync(nsz, 0, ((size_t)nleaf + 1) * sizeof(int64_t), s));
    k_near_sizes<<<grid_for(nleaf), kT, 0, s>>>(h.near_ptr, h.near_src, h.box_start, h.box_end, offL, nleaf, nsz);
    H3D_LAUNCH_CHECK();
    h.near_interactions = scan_exclusive(nsz, nszp, nleaf + 1, s, tmp);
}

bool update_points(Handle &h, const double *points, cudaStream_t s, Arena &tmp) {
    const int64_t n = h.N;
    int *flags = tmp.get<int>(1);
    H3D_CUDA(cudaMemsetAsync(flags, 0, sizeof(int), s));
    k_points_differ<<<grid_for(n), kT, 0, s>>>(points, h.perm, n, h.px, h.py, h.pz, flags);
    H3D_LAUNCH_CHECK();
    const int f = read_scalar(flags, s);
    tmp.free_one(flags);
    if (f & 2) fail(H3D_ERR_DOMAIN);
    if (!(f & 1)) return false;
    k_gather_points<<<grid_for(n), kT, 0, s>>>(points, h.perm, n, h.px, h.py, h.pz);
    H3D_LAUNCH_CHECK();
    const double hL = h.side / (double)(1 << h.L);
    k_local_coords<<<grid_for(n), kT, 0, s>>>(h.px, h.py, h.pz, h.point_leaf, h.box_key, h.box_off[h.L], h.L,
                                                h.lo[0], h.lo[1], h.lo[2], hL, n, h.ploc, h.ploc_lo);
    H3D_LAUNCH_CHECK();
    return true;
}

void unsorted_points(const Handle &h, double *out, cudaStream_t s) {
    k_scatter_points<<<grid_for(h.N), kT, 0, s>>>(h.px, h.py, h.pz, h.perm, h.N, out);
    H3D_LAUNCH_CHECK();
}

}  // namespace h3d
