// primitives.cu -- exclusive scan and stable LSD radix sort for sm_103a.
//
// The radix sort orders the Morton keys of the octree (paper §3.2: the
// octree is built over key-sorted particles) and the interaction lists.
// It takes 8-bit digits: one launch counts the digits of all passes, then
// each pass is one launch (see k_os_scatter); equal digits keep their input
// order, so equal keys keep the order of their values.
#include <algorithm>
#include <atomic>
#include <cstdlib>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

constexpr int kSortThreads = 256;
constexpr int kSortItems = kRadixTile / kSortThreads;
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

// ---- one-sweep LSD radix sort
// One launch counts the digits of every pass at once (the digit counts of a
// pass do not depend on the order the earlier passes leave).  Each pass is
// then one launch: a block takes the next tile in claim order, ranks its keys
// stably (warp by warp, round by round), publishes its per-digit counts, adds
// up the counts of the tiles before it by looking back through their
// published words (decoupled look-back), and writes its keys out grouped by
// digit through shared memory, so that runs of equal digits leave as
// contiguous stores.  A status word is (flag << 32) | count, flag 1 = this
// tile's own count, 2 = the inclusive prefix through this tile.  A block
// waits only on tiles claimed before its own, whose blocks are running and
// publish their own counts before they wait on anything, so every wait
// ends.  The waits are bounded all the same: a block one of whose waits
// gives up counts the digits of all earlier tiles from the input instead
// (exact, slow) and sets kErrSortWait in the error word.  The bound is
// max_polls reads of the awaited word (kOsWait unless the environment
// variable FMM_SORT_POLLS sets it); 0 makes every look-back give up at once,
// which runs the recount in every tile after the first.
constexpr uint64_t kStAgg = 1ull << 32, kStIncl = 2ull << 32;
constexpr int kOsWait = 1 << 20;                 // polls before a wait gives up

__global__ void __launch_bounds__(kSortThreads)
k_os_hist(const uint64_t *keys, int64_t n, int passes, uint32_t *ghist, uint64_t *status0,
          int64_t ntiles)
{
    __shared__ uint32_t h[kRadixMaxPasses][256];
    for (int p = 0; p < passes; ++p) h[p][threadIdx.x] = 0;
    // zero the status words of the first pass (the pass k scatter zeroes those of pass k + 1)
    for (int64_t w = blockIdx.x * (int64_t)kSortThreads + threadIdx.x; w < ntiles * 256;
         w += (int64_t)gridDim.x * kSortThreads)
        status0[w] = 0ull;
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)kSortThreads + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * kSortThreads) {
        const uint64_t key = keys[k];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(unsigned)(key >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int p = 0; p < passes; ++p)
        if (h[p][threadIdx.x]) atomicAdd(&ghist[p * 256 + threadIdx.x], h[p][threadIdx.x]);
}

// Exclusive scan over the 256 threads of one value each (kSortThreads == 256).
__device__ __forceinline__ uint32_t scan256(uint32_t v, uint32_t *warp_sums)
{
    uint32_t total;
    return block_exclusive_scan(v, &total, warp_sums);
}

__global__ void __launch_bounds__(kSortThreads)
k_os_scatter(const uint64_t *keys, const uint32_t *vals, uint64_t *okeys, uint32_t *ovals,
             int64_t n, int pass, int passes, const uint32_t *ghist, unsigned *tile_ctr,
             uint64_t *status, uint64_t *status_next, int *err, int max_polls)
{
    extern __shared__ __align__(16) unsigned char os_smem[];
    uint64_t *sk = (uint64_t *)os_smem;                               // [kSortTile]
    uint32_t *sv = (uint32_t *)(sk + kSortTile);                      // [kSortTile]
    uint32_t (*wh)[256] = (uint32_t (*)[256])(sv + kSortTile);        // [kSortWarps][256]
    uint32_t *dst = (uint32_t *)(wh + kSortWarps);                    // [256] output base per digit
    uint32_t *ls = dst + 256;                                         // [256] digit start in the tile
    __shared__ uint32_t warp_sums[32];
    __shared__ int s_tile, s_gave_up;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int shift = 8 * pass;
    if (tid == 0) {
        s_tile = (int)atomicAdd(&tile_ctr[pass], 1u);
        s_gave_up = 0;
    }
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) wh[w][tid] = 0;
    __syncthreads();
    const int64_t tile = s_tile;
    if (pass + 1 < passes) status_next[tile * 256 + tid] = 0ull;
    const int64_t base = tile * kSortTile;
    const int cnt = (int)min((int64_t)kSortTile, n - base);

    // stable ranking inside the tile: warp w owns items [w*512, (w+1)*512) in
    // input order, round i holding items w*512 + 32 i + lane
    uint64_t key[kSortItems];
    uint32_t val[kSortItems], off[kSortItems];
    const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const int e = warp * (kSortItems * 32) + i * 32 + lane;
        const bool valid = e < cnt;
        key[i] = valid ? keys[base + e] : 0ull;
        val[i] = valid ? vals[base + e] : 0u;
    }
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const int e = warp * (kSortItems * 32) + i * 32 + lane;
        const bool valid = e < cnt;
        const unsigned d = valid ? ((unsigned)(key[i] >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (lane == leader && valid) {
            before = wh[warp][d];
            wh[warp][d] = before + __popc(peers);
        }
        before = __shfl_sync(0xffffffffu, before, leader);
        off[i] = before + __popc(peers & lt_mask);
        __syncwarp();
    }
    __syncthreads();
    // digit tid: warps' exclusive offsets, the tile's count, published at once
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t x = wh[w][tid];
        wh[w][tid] = c;
        c += x;
    }
    volatile uint64_t *vs = (volatile uint64_t *)status;
    vs[tile * 256 + tid] = (tile == 0 ? kStIncl : kStAgg) | c;
    // tiles before this one: the exclusive prefix of digit tid
    uint32_t excl = 0;
    bool ok = true;
    for (int64_t j = tile - 1; j >= 0; --j) {
        uint64_t w = vs[j * 256 + tid];
        int polls = 0;
        while ((w >> 32) == 0 && polls < max_polls) {
            if (++polls > 64) __nanosleep(64);
            w = vs[j * 256 + tid];
        }
        if ((w >> 32) == 0 || max_polls == 0) { ok = false; break; }
        excl += (uint32_t)w;
        if ((w >> 32) == 2) break;
    }
    if (!ok) s_gave_up = 1;
    else if (tile > 0) vs[tile * 256 + tid] = kStIncl | (excl + c);
    __syncthreads();
    if (s_gave_up) {
        // a wait gave up: count the digits of every earlier tile from the
        // input instead (slow, still exact), publish, and flag the event
        dst[tid] = 0;
        __syncthreads();
        for (int64_t k = tid; k < base; k += kSortThreads)
            atomicAdd(&dst[(unsigned)(keys[k] >> shift) & 255u], 1u);
        __syncthreads();
        excl = dst[tid];
        vs[tile * 256 + tid] = kStIncl | (excl + c);
        if (tid == 0) atomicOr(err, kErrSortWait);
        __syncthreads();
    }
    const uint32_t lstart = scan256(c, warp_sums);           // digit start inside the tile
    __syncthreads();
    const uint32_t gstart = scan256(ghist[pass * 256 + tid], warp_sums);
    dst[tid] = gstart + excl - lstart;
    ls[tid] = lstart;
    __syncthreads();
    // the tile in digit order in shared memory, then out: element q of that
    // order goes to dst[digit] + q, so equal digits leave as contiguous runs
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const int e = warp * (kSortItems * 32) + i * 32 + lane;
        if (e < cnt) {
            const unsigned d = (unsigned)(key[i] >> shift) & 255u;
            const uint32_t q = ls[d] + wh[warp][d] + off[i];
            sk[q] = key[i];
            sv[q] = val[i];
        }
    }
    __syncthreads();
    for (int q = tid; q < cnt; q += kSortThreads) {
        const uint64_t k = sk[q];
        const uint32_t pos = dst[(unsigned)(k >> shift) & 255u] + (uint32_t)q;
        okeys[pos] = k;
        ovals[pos] = sv[q];
    }
}

constexpr size_t kOsSmem = (size_t)kSortTile * 12 + (size_t)kSortWarps * 256 * 4 + 2 * 256 * 4;

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
    return 4 * (size_t)radix_hist_words(n);
}

void radix_sort_prepare()
{
    // once per device; threads that race here both set the same value, which is harmless
    static std::atomic<bool> attr_set[64];
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = -1;
    }
    if (dev < 0 || dev >= 64 || !attr_set[dev].load(std::memory_order_acquire)) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, k_os_hist) != cudaSuccess) cudaGetLastError();
        const bool ok = cudaFuncSetAttribute(k_os_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kOsSmem) == cudaSuccess;
        if (!ok) cudaGetLastError();
        if (ok && dev >= 0 && dev < 64) attr_set[dev].store(true, std::memory_order_release);
    }
}

void radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys2, uint32_t *vals2, int64_t n,
                      int end_bit, uint32_t *hist, int *err, cudaStream_t st, int64_t *launches,
                      bool counted)
{
    if (n <= 1) return;
    const int passes = std::min((end_bit + 7) / 8, kRadixMaxPasses);
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    // hist: digit counts [passes][256], tile counters [16], two status areas [ntiles][256]
    uint32_t *ghist = hist, *ctr = hist + kRadixMaxPasses * 256;
    uint64_t *status[2] = {(uint64_t *)(hist + kRadixHead), (uint64_t *)(hist + kRadixHead) + ntiles * 256};
    radix_sort_prepare();
    int max_polls = kOsWait;
    if (const char *env = getenv("FMM_SORT_POLLS")) max_polls = std::max(0, atoi(env));
    if (!counted) {
        cudaMemsetAsync(hist, 0, 4 * (size_t)kRadixHead, st);
        const unsigned hgrid = (unsigned)std::min<int64_t>((n + kSortThreads - 1) / kSortThreads,
                                                           4 * (int64_t)sm_count());
        k_os_hist<<<hgrid, kSortThreads, 0, st>>>(keys, n, passes, ghist, status[0], ntiles);
        ++*launches;
    }
    uint64_t *ka = keys, *kb = keys2;
    uint32_t *va = vals, *vb = vals2;
    for (int p = 0; p < passes; ++p) {
        k_os_scatter<<<(unsigned)ntiles, kSortThreads, kOsSmem, st>>>(
            ka, va, kb, vb, n, p, passes, ghist, ctr, status[p & 1], status[(p + 1) & 1], err, max_polls);
        ++*launches;
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (passes & 1) {
        cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
    }
}

}  // namespace fmm
