// h3d_util.cu -- device prefix sums and a stable LSD radix sort of (key, value)
// pairs, the building blocks of the octree construction (Sec. 2.1).
#include "h3d_internal.cuh"

namespace h3d {

int64_t &fail_alloc_countdown() {
    static int64_t countdown = -1;
    return countdown;
}

int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// ---------------------------------------------------------------------------
// exclusive scan: tiles of 2048 values (256 threads x 8), tile sums scanned
// recursively, then added back.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

template <class TIn>
__global__ void k_scan_tiles(const TIn *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                             int64_t *__restrict__ tile_sums) {
    __shared__ int64_t wsum[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t idx = base + k;
        v[k] = idx < n ? (int64_t)in[idx] : 0;
        s += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = warp_incl_scan(s);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < kScanThreads / 32 ? wsum[lane] : 0;
        w = warp_incl_scan(w);
        if (lane < kScanThreads / 32) wsum[lane] = w;
    }
    __syncthreads();
    int64_t run = incl - s + (warp > 0 ? wsum[warp - 1] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t idx = base + k;
        if (idx < n) out[idx] = run;
        run += v[k];
    }
    if (threadIdx.x == kScanThreads - 1) tile_sums[blockIdx.x] = run;
}

__global__ void k_scan_add(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ pref) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const int64_t add = pref[blockIdx.x];
    for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
        int64_t idx = base + k;
        if (idx < n) out[idx] += add;
    }
}

template <class TIn>
static void scan_rec(const TIn *in, int64_t *out, int64_t n, int64_t *d_total, cudaStream_t s, Arena &tmp) {
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    int64_t *sums = tmp.get<int64_t>((size_t)ntiles);
    k_scan_tiles<TIn><<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, out, n, sums);
    H3D_LAUNCH_CHECK();
    if (ntiles == 1) {
        H3D_CUDA(cudaMemcpyAsync(d_total, sums, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    } else {
        int64_t *pref = tmp.get<int64_t>((size_t)ntiles);
        scan_rec<int64_t>(sums, pref, ntiles, d_total, s, tmp);
        k_scan_add<<<(unsigned)ntiles, kScanThreads, 0, s>>>(out, n, pref);
        H3D_LAUNCH_CHECK();
    }
}

template <class TIn>
static int64_t scan_impl(const TIn *in, int64_t *out, int64_t n, cudaStream_t s, Arena &tmp) {
    if (n <= 0) return 0;
    int64_t *d_total = tmp.get<int64_t>(1);
    scan_rec<TIn>(in, out, n, d_total, s, tmp);
    return read_scalar(d_total, s);
}

int64_t scan_exclusive(const int *in, int64_t *out, int64_t n, cudaStream_t s, Arena &tmp) {
    return scan_impl<int>(in, out, n, s, tmp);
}
int64_t scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s, Arena &tmp) {
    return scan_impl<int64_t>(in, out, n, s, tmp);
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits.  Per pass: per-tile digit histograms
// (digit-major), an exclusive scan over (digit, tile), and a stable scatter in
// which every tile ranks its items in input order (warp match + per-warp
// counts in shared memory).
constexpr int kRsThreads = 256;
constexpr int kRsRounds = 8;
constexpr int kRsTile = kRsThreads * kRsRounds;

__global__ void k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int shift, int *__restrict__ counts,
                          int ntiles) {
    __shared__ int hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsRounds; ++r) {
        int64_t idx = base + r * kRsThreads + threadIdx.x;
        if (idx < n) atomicAdd(&hist[(unsigned)(keys[idx] >> shift) & 255u], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = hist[threadIdx.x];
}

__global__ void k_rs_scatter(const uint64_t *__restrict__ kin, const int *__restrict__ vin,
                             uint64_t *__restrict__ kout, int *__restrict__ vout, int64_t n, int shift,
                             const int64_t *__restrict__ offs, int ntiles) {
    __shared__ int64_t base[256];
    __shared__ int wcnt[kRsThreads / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < kRsRounds; ++r) {
#pragma unroll
        for (int w = 0; w < kRsThreads / 32; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const int64_t idx = (int64_t)blockIdx.x * kRsTile + r * kRsThreads + tid;
        const bool valid = idx < n;
        uint64_t key = 0;
        int val = 0;
        unsigned d = 256u;
        if (valid) {
            key = kin[idx];
            val = vin[idx];
            d = (unsigned)(key >> shift) & 255u;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt_mask);
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
        for (int w = 0; w < kRsThreads / 32; ++w) tot += wcnt[w][tid];
        base[tid] += tot;
        __syncthreads();
    }
}

void radix_sort_pairs(uint64_t *keys, int *vals, int64_t n, int key_bits, cudaStream_t s, Arena &tmp) {
    if (n <= 1) return;
    const int ntiles = (int)((n + kRsTile - 1) / kRsTile);
    uint64_t *k2 = tmp.get<uint64_t>((size_t)n);
    int *v2 = tmp.get<int>((size_t)n);
    int *counts = tmp.get<int>((size_t)ntiles * 256);
    int64_t *offs = tmp.get<int64_t>((size_t)ntiles * 256);
    uint64_t *ka = keys, *kb = k2;
    int *va = vals, *vb = v2;
    const int passes = (key_bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        k_rs_hist<<<ntiles, kRsThreads, 0, s>>>(ka, n, shift, counts, ntiles);
        H3D_LAUNCH_CHECK();
        scan_exclusive(counts, offs, (int64_t)ntiles * 256, s, tmp);
        k_rs_scatter<<<ntiles, kRsThreads, 0, s>>>(ka, va, kb, vb, n, shift, offs, ntiles);
        H3D_LAUNCH_CHECK();
        uint64_t *tk = ka; ka = kb; kb = tk;
        int *tv = va; va = vb; vb = tv;
    }
    if (ka != keys) {
        H3D_CUDA(cudaMemcpyAsync(keys, ka, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        H3D_CUDA(cudaMemcpyAsync(vals, va, (size_t)n * sizeof(int), cudaMemcpyDeviceToDevice, s));
    }
}

}  // namespace h3d
