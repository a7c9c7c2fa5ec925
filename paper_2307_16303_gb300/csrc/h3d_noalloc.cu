// h3d_noalloc.cu -- Morton keys and Morton order of a point set without any
// memory allocation, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running under an allocator that
// forbids it (a fixed memory pool handed out by a host application), code
// inside a region where allocation would break an external memory budget, or
// plugins that only receive pre-allocated buffers.  For them this entry point
// computes what the first two steps of h3d_build compute -- one 63-bit Morton
// key per point and the stable order of the points by (key, original index) --
// using a fixed scratch area that lives in this file as a static device array.
//
// The scratch array is part of the library image: every GPU that loads the
// library holds it until the process exits.  All calls share it, so calls that
// overlap on the GPU (for example on two streams at once) race on it; callers
// must serialise them.  The array keeps the contents of the last call; what
// must start at zero (the error word) is cleared by every call.
#include <cmath>
#include <mutex>

#include "h3d_internal.cuh"

namespace {

constexpr int64_t kMaxPoints = H3D_NOALLOC_MAX_POINTS;
constexpr int kThreads = 256;
constexpr int kRounds = 8;
constexpr int kTile = kThreads * kRounds;
constexpr int64_t kMaxTiles = (kMaxPoints + kTile - 1) / kTile;
constexpr int64_t kCounts = kMaxTiles * 256;

// scratch layout (bytes): keys | values | per-tile digit counts | offsets | error word
constexpr size_t kOffKeys = 0;
constexpr size_t kOffVals = kOffKeys + (size_t)kMaxPoints * 8;
constexpr size_t kOffCounts = kOffVals + (size_t)kMaxPoints * 4;
constexpr size_t kOffOffs = kOffCounts + (size_t)kCounts * 4;
constexpr size_t kOffErr = kOffOffs + (size_t)kCounts * 8;
constexpr size_t kScratchBytes = kOffErr + 256;
static_assert(kScratchBytes <= (size_t)H3D_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the declared size");

__device__ __align__(256) unsigned char g_noalloc_scratch[H3D_NOALLOC_SCRATCH_BYTES];

__device__ __forceinline__ uint64_t spread21(uint64_t v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__global__ void k_na_keys(const double *__restrict__ pts, int64_t n, double lo0, double lo1, double lo2, double side,
                          uint64_t *__restrict__ keys, int *__restrict__ idx, int *__restrict__ err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
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
        const uint64_t q = (uint64_t)floor(__dmul_rn(t, 2097152.0));
        c[d] = q > 2097151ull ? 2097151ull : q;
    }
    if (bad) atomicOr(err, 1);
    keys[i] = (spread21(c[0]) << 2) | (spread21(c[1]) << 1) | spread21(c[2]);
    idx[i] = (int)i;
}

__global__ void k_na_hist(const uint64_t *__restrict__ keys, int64_t n, int shift, int *__restrict__ counts,
                          int ntiles) {
    __shared__ int hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    for (int r = 0; r < kRounds; ++r) {
        const int64_t i = (int64_t)blockIdx.x * kTile + r * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&hist[(unsigned)(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = hist[threadIdx.x];
}

// exclusive scan of m <= kCounts ints by one CTA of 1024 threads
__global__ void __launch_bounds__(1024) k_na_scan(const int *__restrict__ in, int64_t *__restrict__ out, int m) {
    __shared__ int64_t part[1024];
    const int per = (m + 1023) / 1024;
    const int b = threadIdx.x * per, e = min(m, b + per);
    int64_t s = 0;
    for (int i = b; i < e; ++i) s += in[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int64_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = part[threadIdx.x] - s;
    for (int i = b; i < e; ++i) {
        out[i] = run;
        run += in[i];
    }
}

__global__ void k_na_scatter(const uint64_t *__restrict__ kin, const int *__restrict__ vin, uint64_t *__restrict__ kout,
                             int *__restrict__ vout, int64_t n, int shift, const int64_t *__restrict__ offs,
                             int ntiles) {
    __shared__ int64_t base[256];
    __shared__ int wcnt[kThreads / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kRounds; ++r) {
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const int64_t i = (int64_t)blockIdx.x * kTile + r * kThreads + tid;
        const bool valid = i < n;
        uint64_t key = 0;
        int val = 0;
        unsigned d = 256u;
        if (valid) {
            key = kin[i];
            val = vin[i];
            d = (unsigned)(key >> shift) & 255u;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int64_t pos = base[d] + rank;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        int tot = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) tot += wcnt[w][tid];
        base[tid] += tot;
        __syncthreads();
    }
}

// Device address of the scratch array, resolved once per device.
std::mutex g_mu;
void *g_addr[64] = {nullptr};

h3d_status scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return H3D_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return H3D_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return H3D_OK;
}

// true for memory the GPU reaches as device memory (cudaMalloc'ed or managed);
// asks the runtime only, allocates nothing
bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" h3d_status h3d_morton_order_noalloc(const double *points, int64_t N, const double *lo, double side,
                                               uint64_t *keys_out, int *perm_out, void *stream) {
    if (!points || !lo || !keys_out || !perm_out || N < 1) return H3D_ERR_ARG;
    if (N > kMaxPoints) return H3D_ERR_ARG;  // beyond the fixed scratch: rejected, never truncated
    // host buffers would fault the kernels: rejected before any launch
    if (!is_device_ptr(points) || !is_device_ptr(keys_out) || !is_device_ptr(perm_out)) return H3D_ERR_ARG;
    if (!(side > 0.0) || !std::isfinite(side)) return H3D_ERR_ARG;
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(lo[d])) return H3D_ERR_ARG;
    void *base = nullptr;
    h3d_status st = scratch_address(&base);
    if (st != H3D_OK) return st;
    unsigned char *sc = static_cast<unsigned char *>(base);
    uint64_t *skeys = reinterpret_cast<uint64_t *>(sc + kOffKeys);
    int *svals = reinterpret_cast<int *>(sc + kOffVals);
    int *counts = reinterpret_cast<int *>(sc + kOffCounts);
    int64_t *offs = reinterpret_cast<int64_t *>(sc + kOffOffs);
    int *err = reinterpret_cast<int *>(sc + kOffErr);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int ntiles = (int)((N + kTile - 1) / kTile);
    const unsigned nb = (unsigned)((N + kThreads - 1) / kThreads);
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return H3D_ERR_CUDA;
    }
    k_na_keys<<<nb, kThreads, 0, s>>>(points, N, lo[0], lo[1], lo[2], side, keys_out, perm_out, err);
    // 8 passes of 8 bits; even count, so the result ends in the caller's buffers
    uint64_t *ka = keys_out, *kb = skeys;
    int *va = perm_out, *vb = svals;
    for (int p = 0; p < 8; ++p) {
        k_na_hist<<<ntiles, kThreads, 0, s>>>(ka, N, 8 * p, counts, ntiles);
        k_na_scan<<<1, 1024, 0, s>>>(counts, offs, ntiles * 256);
        k_na_scatter<<<ntiles, kThreads, 0, s>>>(ka, va, kb, vb, N, 8 * p, offs, ntiles);
        uint64_t *tk = ka; ka = kb; kb = tk;
        int *tv = va; va = vb; vb = tv;
    }
    if (cudaGetLastError() != cudaSuccess) return H3D_ERR_CUDA;
    int herr = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return H3D_ERR_CUDA;
    }
    return herr ? H3D_ERR_DOMAIN : H3D_OK;
}
