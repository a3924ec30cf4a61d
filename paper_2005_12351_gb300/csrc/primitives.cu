// primitives.cu -- exclusive scan and stable LSD radix sort for sm_103a.
//
// The radix sort orders the Morton keys of the octree (paper §3.2: the
// octree is built over key-sorted particles) and the interaction lists.
// Each 8-bit pass is three launches: per-tile digit histograms, one
// exclusive scan of the digit-major histogram, and a stable scatter in which
// every tile ranks its keys round by round with __match_any_sync, so equal
// digits keep their input order (ties are broken by the original index).
#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSortWarps = kSortThreads / 32;

// Exclusive scan of one value per thread across the block; *total gets the sum.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total,
                                                         uint32_t *warp_sums)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nwarps ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    uint32_t pre = warp == 0 ? 0u : warp_sums[warp - 1];
    *total = warp_sums[nwarps - 1];
    return pre + x - v;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_tiles(const uint32_t *in, uint32_t *out, uint32_t *tile_sums, int64_t n)
{
    __shared__ uint32_t warp_sums[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t k = base + i;
        v[i] = k < n ? in[k] : 0u;
        sum += v[i];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(sum, &total, warp_sums);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t k = base + i;
        if (k < n) out[k] = run;
        run += v[i];
    }
    if (threadIdx.x == 0 && tile_sums) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_add(uint32_t *out, const uint32_t *tile_offsets, int64_t n)
{
    const uint32_t add = tile_offsets[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
        int64_t k = base + i;
        if (k < n) out[k] += add;
    }
}

__global__ void __launch_bounds__(kSortThreads)
k_radix_hist(const uint64_t *keys, int64_t n, int shift, uint32_t *hist, int ntiles)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int i = 0; i < kSortItems; ++i) {
        int64_t k = base + (int64_t)i * kSortThreads + threadIdx.x;
        if (k < n) atomicAdd(&h[(unsigned)(keys[k] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads)
k_radix_scatter(const uint64_t *keys, const uint32_t *vals, uint64_t *okeys, uint32_t *ovals,
                int64_t n, int shift, const uint32_t *hist_scan, int ntiles)
{
    __shared__ uint32_t run[256];
    __shared__ uint32_t wcnt[kSortWarps][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    run[tid] = hist_scan[(int64_t)tid * ntiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int i = 0; i < kSortItems; ++i) {
        const int64_t k = base + (int64_t)i * kSortThreads + tid;
        const bool valid = k < n;
        const uint64_t key = valid ? keys[k] : 0ull;
        const uint32_t val = valid ? vals[k] : 0u;
        const unsigned d = valid ? ((unsigned)(key >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned rank = __popc(peers & lt_mask);
        if (valid && (__ffs(peers) - 1) == lane) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {   // digit `tid`: exclusive prefix over the warps of this round
            uint32_t r = run[tid];
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = r;
                r += c;
            }
            run[tid] = r;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = wcnt[warp][d] + rank;
            okeys[pos] = key;
            ovals[pos] = val;
        }
        __syncthreads();
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) wcnt[w][tid] = 0;
        __syncthreads();
    }
}

}  // namespace

size_t scan_scratch_bytes(int64_t n)
{
    size_t total = 0;
    int64_t m = n;
    while (m > kScanTile) {
        m = (m + kScanTile - 1) / kScanTile;
        total += 2 * (size_t)m;            // tile sums + their scan
    }
    return (total + 64) * sizeof(uint32_t);
}

void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *scratch,
                        cudaStream_t st, int64_t *launches)
{
    if (n <= 0) return;
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        k_scan_tiles<<<1, kScanThreads, 0, st>>>(in, out, nullptr, n);
        ++*launches;
        return;
    }
    uint32_t *sums = scratch, *sums_scan = scratch + tiles;
    k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, sums, n);
    exclusive_scan_u32(sums, sums_scan, tiles, scratch + 2 * tiles, st, launches);
    k_scan_add<<<(unsigned)tiles, 256, 0, st>>>(out, sums_scan, n);
    *launches += 2;
}

size_t radix_hist_bytes(int64_t n)
{
    const int64_t tiles = (n + kSortTile - 1) / kSortTile;
    return (size_t)(256 * (tiles > 0 ? tiles : 1)) * sizeof(uint32_t);
}

void radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys2, uint32_t *vals2, int64_t n,
                      int end_bit, uint32_t *hist, uint32_t *scan_scratch, cudaStream_t st,
                      int64_t *launches)
{
    if (n <= 1) return;
    const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    uint64_t *ka = keys, *kb = keys2;
    uint32_t *va = vals, *vb = vals2;
    int passes = 0;
    for (int shift = 0; shift < end_bit; shift += 8, ++passes) {
        k_radix_hist<<<ntiles, kSortThreads, 0, st>>>(ka, n, shift, hist, ntiles);
        exclusive_scan_u32(hist, hist, (int64_t)256 * ntiles, scan_scratch, st, launches);
        k_radix_scatter<<<ntiles, kSortThreads, 0, st>>>(ka, va, kb, vb, n, shift, hist, ntiles);
        *launches += 2;
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    if (passes & 1) {
        cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
    }
}

}  // namespace fmm
