// tree.cu -- octree and interaction lists on the GPU (paper §3.2).
//
// Root box: lo = per-axis minimum; side = the smallest power of two not below
// the largest extent.  Integer coordinates q = min(floor((x - lo) * 2^21 /
// side), 2^21 - 1) are interleaved (x highest) into 63-bit Morton keys and
// sorted stably.  Cells are built breadth-first: a cell splits while it holds
// more than n_crit particles and its level is below 21; empty octants are
// not created, so cells come out in (level, Morton prefix) order.
//
// Lists come from the dual-tree traversal of §3.2 run as a breadth-first
// frontier of cell pairs.  MAC (Eq. (13)) with r = half the cell side,
// evaluated exactly in integer units of the finest half-cell; when it fails:
// two leaves -> P2P, one leaf -> open the other, else open the larger cell
// (the target on a tie); a self pair opens into all ordered child pairs.
#include <algorithm>
#include <cmath>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

__device__ __forceinline__ unsigned long long ordered_bits(double x)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_ordered_bits(unsigned long long b)
{
    b = (b >> 63) ? (b & 0x7fffffffffffffffull) : ~b;
    return __longlong_as_double((long long)b);
}

__global__ void k_box_init(unsigned long long *box)
{
    int i = threadIdx.x;
    if (i < 3) box[i] = ~0ull;            // running minimum
    else if (i < 6) box[i] = 0ull;        // running maximum
}

__global__ void k_bbox(const double *pos, int64_t n, unsigned long long *box, int *err)
{
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double x = pos[3 * i + d];
            if (!isfinite(x)) bad = true;
            unsigned long long b = ordered_bits(x);
            mn[d] = b < mn[d] ? b : mn[d];
            mx[d] = b > mx[d] ? b : mx[d];
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long a = __shfl_xor_sync(0xffffffffu, mn[d], o);
            unsigned long long b = __shfl_xor_sync(0xffffffffu, mx[d], o);
            mn[d] = a < mn[d] ? a : mn[d];
            mx[d] = b > mx[d] ? b : mx[d];
        }
    }
    // the block's warps through shared memory, then six atomics per block
    __shared__ unsigned long long s_mm[6][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) { s_mm[d][warp] = mn[d]; s_mm[3 + d][warp] = mx[d]; }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int d = threadIdx.x;
        unsigned long long v = s_mm[d][0];
        for (int w = 1; w < nw; ++w) v = d < 3 ? (s_mm[d][w] < v ? s_mm[d][w] : v) : (s_mm[d][w] > v ? s_mm[d][w] : v);
        if (d < 3) atomicMin(&box[d], v); else atomicMax(&box[d], v);
    }
    if (bad) atomicOr(err, kErrNonFinite);
}

// box_out = (lo_x, lo_y, lo_z, side)
__global__ void k_box_final(const unsigned long long *box, double *box_out)
{
    double lo[3], ext = 0.0;
    for (int d = 0; d < 3; ++d) {
        lo[d] = from_ordered_bits(box[d]);
        double e = __dsub_rn(from_ordered_bits(box[3 + d]), lo[d]);
        ext = e > ext ? e : ext;
    }
    double side = 1.0;
    if (ext > 0.0 && isfinite(ext)) {
        int e2;
        double m = frexp(ext, &e2);        // ext = m 2^e2, m in [0.5, 1)
        side = ldexp(1.0, m == 0.5 ? e2 - 1 : e2);
    }
    box_out[0] = lo[0]; box_out[1] = lo[1]; box_out[2] = lo[2]; box_out[3] = side;
}

__device__ __forceinline__ uint64_t spread3(uint64_t x)
{
    x &= 0x1fffffull;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

// floor(d 2^k) for a double d >= 0 and 2^k a power of two, clamped to the
// grid (the product is exact, so this is floor((x - lo) scale) of the
// definition), from d's bits: one FP64 operation per coordinate, the rest
// integer arithmetic.
__device__ __forceinline__ uint64_t grid_coord(double d, int k)
{
    const uint64_t b = (uint64_t)__double_as_longlong(d);
    const int ef = (int)((b >> 52) & 0x7ff);
    // d = m 2^(e - 1075), subnormals with e = 1 and no implicit bit
    const uint64_t m = (b & ((1ull << 52) - 1)) | (ef ? (1ull << 52) : 0ull);
    const int sh = (ef ? ef : 1) - 1075 + k;        // d 2^k = m 2^sh
    const uint64_t top = (uint64_t)((1 << kLevels) - 1);
    if (sh >= 0) return sh > 11 ? top : ((m << sh) > top ? top : (m << sh));
    return sh <= -64 ? 0 : ((m >> -sh) > top ? top : (m >> -sh));
}

// The keys, and for the radix sort that follows the counts of every 8-bit
// digit of them (per block in shared memory, then one atomic per digit and
// block) and the zeroed status words of its first pass.
__global__ void __launch_bounds__(256)
k_keys(const double *pos, int64_t n, const double *box, uint64_t *keys, uint32_t *idx,
       uint32_t *ghist, uint64_t *status0, int64_t nstatus)
{
    __shared__ uint32_t h[kRadixMaxPasses][256];
#pragma unroll
    for (int p = 0; p < kRadixMaxPasses; ++p) h[p][threadIdx.x] = 0;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nstatus;
         w += (int64_t)gridDim.x * blockDim.x)
        status0[w] = 0ull;
    __syncthreads();
    const int k = kLevels - ilogb(box[3]);          // scale = 2^kLevels / side = 2^k
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t q[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) q[d] = grid_coord(__dsub_rn(pos[3 * i + d], box[d]), k);
        const uint64_t key = spread3(q[0]) << 2 | spread3(q[1]) << 1 | spread3(q[2]);
        keys[i] = key;
        idx[i] = (uint32_t)i;
#pragma unroll
        for (int p = 0; p < kRadixMaxPasses; ++p) atomicAdd(&h[p][(unsigned)(key >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < kRadixMaxPasses; ++p)
        if (h[p][threadIdx.x]) atomicAdd(&ghist[p * 256 + threadIdx.x], h[p][threadIdx.x]);
}

// ---- systems (a forest of independent octrees, one root per system)
__global__ void k_sys_of(const int64_t *off, int nsys, int64_t n, int32_t *sys_of)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = nsys - 1;                 // last system whose start is <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    sys_of[i] = lo;
}

__global__ void k_box_init_seg(unsigned long long *box, int nsys)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6 * nsys) return;
    box[i] = (i % 6) < 3 ? ~0ull : 0ull;
}

// Per-system min/max.  A warp whose particles all belong to one system
// reduces with shuffles first; mixed warps fall back to per-lane atomics.
__global__ void k_bbox_seg(const double *pos, int64_t n, const int32_t *sys_of,
                           unsigned long long *box, int *err)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool valid = i < n;
    const int s = valid ? sys_of[i] : -1;
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
    bool bad = false;
    if (valid) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double x = pos[3 * i + d];
            if (!isfinite(x)) bad = true;
            mn[d] = mx[d] = ordered_bits(x);
        }
    }
    const int s0 = __shfl_sync(0xffffffffu, s, 0);
    const bool uniform = __all_sync(0xffffffffu, s == s0);
    if (uniform) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                unsigned long long a = __shfl_xor_sync(0xffffffffu, mn[d], o);
                unsigned long long b = __shfl_xor_sync(0xffffffffu, mx[d], o);
                mn[d] = a < mn[d] ? a : mn[d];
                mx[d] = b > mx[d] ? b : mx[d];
            }
        if ((threadIdx.x & 31) == 0 && s0 >= 0)
            for (int d = 0; d < 3; ++d) {
                atomicMin(&box[6 * s0 + d], mn[d]);
                atomicMax(&box[6 * s0 + 3 + d], mx[d]);
            }
    } else if (valid) {
        for (int d = 0; d < 3; ++d) {
            atomicMin(&box[6 * s + d], mn[d]);
            atomicMax(&box[6 * s + 3 + d], mx[d]);
        }
    }
    if (bad) atomicOr(err, kErrNonFinite);
}

// box_out[4 s .. 4 s + 3] = (lo_x, lo_y, lo_z, side) of system s; empty systems get side 1
__global__ void k_box_final_seg(const unsigned long long *box, int nsys, double *box_out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    const unsigned long long *b = box + 6 * s;
    if (b[0] == ~0ull) {                       // no particles
        box_out[4 * s] = box_out[4 * s + 1] = box_out[4 * s + 2] = 0.0;
        box_out[4 * s + 3] = 1.0;
        return;
    }
    double lo[3], ext = 0.0;
    for (int d = 0; d < 3; ++d) {
        lo[d] = from_ordered_bits(b[d]);
        const double e = __dsub_rn(from_ordered_bits(b[3 + d]), lo[d]);
        ext = e > ext ? e : ext;
    }
    double side = 1.0;
    if (ext > 0.0 && isfinite(ext)) {
        int e2;
        const double m = frexp(ext, &e2);
        side = ldexp(1.0, m == 0.5 ? e2 - 1 : e2);
    }
    box_out[4 * s] = lo[0]; box_out[4 * s + 1] = lo[1]; box_out[4 * s + 2] = lo[2];
    box_out[4 * s + 3] = side;
}

__global__ void k_keys_seg(const double *pos, int64_t n, const int32_t *sys_of,
                           const double *box, uint64_t *keys, uint32_t *idx)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *bx = box + 4 * sys_of[i];
    const double scale = ldexp(1.0, kLevels) / bx[3];
    uint64_t q[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double u = floor(__dmul_rn(__dsub_rn(pos[3 * i + d], bx[d]), scale));
        uint64_t v = (uint64_t)u;
        q[d] = v > (uint64_t)((1 << kLevels) - 1) ? (uint64_t)((1 << kLevels) - 1) : v;
    }
    keys[i] = spread3(q[0]) << 2 | spread3(q[1]) << 1 | spread3(q[2]);
    idx[i] = (uint32_t)i;
}

// after the key sort: secondary key = system of each element, and a copy of
// the sorted keys by original index for the final re-gather
__global__ void k_sys_keys(const uint64_t *keys, const uint32_t *idx, const int32_t *sys_of,
                           int64_t n, uint64_t *skeys, uint64_t *key_of)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    skeys[k] = (uint64_t)sys_of[idx[k]];
    key_of[idx[k]] = keys[k];
}

__global__ void k_regather_keys(const uint64_t *key_of, const uint32_t *idx, int64_t n,
                                uint64_t *keys)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) keys[k] = key_of[idx[k]];
}

__global__ void k_gather(const double *pos, const double *mom, int nS, const uint32_t *perm,
                         int64_t n, double *px, double *py, double *pz, double *S, int32_t *perm_out)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t o = perm[k];
    px[k] = pos[3 * o];
    py[k] = pos[3 * o + 1];
    pz[k] = pos[3 * o + 2];
    for (int a = 0; a < nS; ++a) S[k * nS + a] = mom[o * nS + a];
    perm_out[k] = (int32_t)o;
}

struct CellArrays {
    int32_t *level, *parent, *child, *nchild, *begin, *end, *cx, *cy, *cz, *sys;
};

__global__ void k_roots(CellArrays c, const int64_t *off, int nsys)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    c.level[s] = 0; c.parent[s] = -1; c.begin[s] = (int32_t)off[s]; c.end[s] = (int32_t)off[s + 1];
    c.cx[s] = c.cy[s] = c.cz[s] = 0;
    c.sys[s] = s;
}

__global__ void k_root_pairs(int2 *front, int nsys, unsigned *nf0)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsys) front[s] = make_int2(s, s);
    if (s == 0) *nf0 = (unsigned)nsys;
}

__device__ __forceinline__ int digit_at(uint64_t key, int level)
{
    return (int)((key >> (3 * (kLevels - level))) & 7ull);
}

// ---- cells, level by level without host round trips: the range of a level's
// cells lives in device words (ctl[kCtlLevel + l] = first cell of level l), so
// the host launches the levels back to back and reads the counts once per
// batch.  A level that would pass the cell capacity sets ctl[kCtlOverflow]
// instead; every later kernel then does nothing and the host rebuilds with
// more room.
constexpr int kCtlOverflow = 0, kCtlLevel = 1, kCtlWords = 32;
constexpr int kLevelBatch = 8;                  // levels launched per host round trip
constexpr int kLevelScanPer = 16;               // child counts per thread of the one-block scan

// child ranges of every (cell of this level, octant), and each cell's child
// count.  When the level has at most as many cells as the grid has warps
// (the shallow levels, whose cells hold many particles) a warp takes a cell:
// its seven groups of four lanes each find one octant boundary by a 5-way
// search (four probes a step); otherwise a thread takes a (cell, octant) and
// binary-searches both ends of its range.
__device__ __forceinline__ int first_digit_ge(const uint64_t *keys, int L, int R, int level, int o)
{
    while (L < R) {
        const int mid = (L + R) >> 1;
        if (digit_at(keys[mid], level) < o) L = mid + 1; else R = mid;
    }
    return L;
}

__global__ void __launch_bounds__(256)
k_level_ranges(CellArrays c, const unsigned *ctl, int level, int ncrit, const uint64_t *keys,
               int32_t *cb, int32_t *ce, uint32_t *cnt)
{
    if (ctl[kCtlOverflow]) return;
    const int lb = (int)ctl[kCtlLevel + level];
    const int ncl = (int)ctl[kCtlLevel + level + 1] - lb;
    const int64_t n8 = 8 * (int64_t)ncl;
    const unsigned lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    if (ncl <= nwarps) {
        const int64_t wi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        if (wi >= ncl) return;
        const int cell = lb + (int)wi;
        const int b = c.begin[cell], e = c.end[cell];
        if (!(e - b > ncrit && level < kLevels)) {
            if (lane < 8) { cb[8 * wi + lane] = b; ce[8 * wi + lane] = b; }
            if (lane == 0) cnt[wi] = 0u;
            return;
        }
        const int g = (int)lane >> 2, q = (int)lane & 3;       // group g finds boundary g + 1
        int bnd = b;
        if (g < 7) {
            const unsigned gm = 0xfu << (4 * g);
            int L = b, R = e;
            while (R - L > 4) {
                const int len = R - L;
                const bool lt = digit_at(keys[L + (int)(((int64_t)(q + 1) * len) / 5)], level + 1) < g + 1;
                const int k = __popc(__ballot_sync(gm, lt) & gm);
                const int nL = k > 0 ? L + (int)(((int64_t)k * len) / 5) + 1 : L;
                const int nR = k < 4 ? L + (int)(((int64_t)(k + 1) * len) / 5) : R;
                L = nL;
                R = nR;
            }
            const bool lt = q < R - L && digit_at(keys[L + q], level + 1) < g + 1;
            bnd = L + __popc(__ballot_sync(gm, lt) & gm);
        }
        const int o = (int)(lane & 7);
        const int bl = __shfl_sync(0xffffffffu, bnd, (4 * (o - 1)) & 31);
        const int bh = __shfl_sync(0xffffffffu, bnd, (4 * o) & 31);
        const int lo_i = o == 0 ? b : bl, hi_i = o == 7 ? e : bh;
        const unsigned m = __ballot_sync(0xffffffffu, lane < 8 && hi_i > lo_i);
        if (lane < 8) { cb[8 * wi + lane] = lo_i; ce[8 * wi + lane] = hi_i; }
        if (lane == 0) cnt[wi] = __popc(m);
        return;
    }
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n8; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = base + threadIdx.x;
        bool flag = false;
        if (t < n8) {
            const int cell = lb + (int)(t >> 3), o = (int)(t & 7);
            const int b = c.begin[cell], e = c.end[cell];
            int lo_i = b, hi_i = b;
            if (e - b > ncrit && level < kLevels) {
                // first index in [b, e) whose child digit is >= o (resp. >= o + 1)
                lo_i = first_digit_ge(keys, b, e, level + 1, o);
                hi_i = first_digit_ge(keys, lo_i, e, level + 1, o + 1);
                flag = hi_i > lo_i;
            }
            cb[t] = lo_i;
            ce[t] = hi_i;
        }
        // a cell's 8 octants are 8 aligned lanes of one warp
        const unsigned m = __ballot_sync(0xffffffffu, flag);
        if (t < n8 && (t & 7) == 0) cnt[t >> 3] = __popc((m >> (lane & ~7u)) & 0xffu);
    }
}

// one block: the first-child offset of every cell of this level (an exclusive
// scan of the child counts) and the next level's range, or the overflow flag
__global__ void __launch_bounds__(1024)
k_level_scan(unsigned *ctl, int level, const uint32_t *cnt, uint32_t *off, int64_t cap)
{
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    if (ctl[kCtlOverflow]) return;
    const int lb = (int)ctl[kCtlLevel + level], le = (int)ctl[kCtlLevel + level + 1];
    const int ncl = le - lb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < ncl; base += kLevelScanPer * (int)blockDim.x) {
        const int i0 = base + kLevelScanPer * (int)threadIdx.x;
        uint32_t v[kLevelScanPer], sum = 0;
        if (i0 + kLevelScanPer <= ncl) {             // whole: 16-byte loads (i0 is a multiple of 16)
#pragma unroll
            for (int k = 0; k < kLevelScanPer; k += 4) {
                const uint4 q = *(const uint4 *)(cnt + i0 + k);
                v[k] = q.x; v[k + 1] = q.y; v[k + 2] = q.z; v[k + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kLevelScanPer; ++k) v[k] = i0 + k < ncl ? cnt[i0 + k] : 0u;
        }
#pragma unroll
        for (int k = 0; k < kLevelScanPer; ++k) sum += v[k];
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = lane < nw ? wsum[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        uint32_t ex = carry + (warp ? wsum[warp - 1] : 0u) + x - sum;
        uint32_t o[kLevelScanPer];
#pragma unroll
        for (int k = 0; k < kLevelScanPer; ++k) {
            o[k] = ex;
            ex += v[k];
        }
        if (i0 + kLevelScanPer <= ncl) {
#pragma unroll
            for (int k = 0; k < kLevelScanPer; k += 4)
                *(uint4 *)(off + i0 + k) = make_uint4(o[k], o[k + 1], o[k + 2], o[k + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < kLevelScanPer; ++k)
                if (i0 + k < ncl) off[i0 + k] = o[k];
        }
        const uint32_t tot = wsum[nw - 1];
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if ((int64_t)le + carry > cap) ctl[kCtlOverflow] = 1u;
        else ctl[kCtlLevel + level + 2] = (unsigned)le + carry;
    }
}

// the children of this level's cells, in (parent, octant) order
__global__ void __launch_bounds__(256)
k_level_write(CellArrays c, const unsigned *ctl, int level, const int32_t *cb, const int32_t *ce,
              const uint32_t *off)
{
    if (ctl[kCtlOverflow]) return;
    const int lb = (int)ctl[kCtlLevel + level], le = (int)ctl[kCtlLevel + level + 1];
    const int64_t n8 = 8 * (int64_t)(le - lb);
    const unsigned lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n8; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = base + threadIdx.x;
        const bool valid = t < n8;
        const bool flag = valid && ce[t] > cb[t];
        const unsigned grp = (__ballot_sync(0xffffffffu, flag) >> (lane & ~7u)) & 0xffu;
        if (!valid) continue;
        const int i = (int)(t >> 3), o = (int)(t & 7), cell = lb + i;
        if (o == 0) {
            const int nch = __popc(grp);
            c.nchild[cell] = nch;
            c.child[cell] = nch ? le + (int)off[i] : -1;
        }
        if (!flag) continue;
        const int ch = le + (int)off[i] + __popc(grp & ((1u << o) - 1u));
        c.level[ch] = level + 1;
        c.parent[ch] = cell;
        c.begin[ch] = cb[t];
        c.end[ch] = ce[t];
        c.cx[ch] = 2 * c.cx[cell] + ((o >> 2) & 1);
        c.cy[ch] = 2 * c.cy[cell] + ((o >> 1) & 1);
        c.cz[ch] = 2 * c.cz[cell] + (o & 1);
        c.sys[ch] = c.sys[cell];
    }
}

__global__ void k_level_init(unsigned *ctl, int nsys)
{
    const int i = threadIdx.x;
    if (i < kCtlWords) ctl[i] = i == kCtlLevel + 1 ? (unsigned)nsys : 0u;
}

// Besides the geometry, each cell gets the packed record the traversal reads
// with one 16-byte load: {cx | level << 21, cy | nchild << 21, cz, child}.
__global__ void k_cell_geometry(CellArrays c, int64_t ncells, const double *box, double *centre,
                                double *half, uint32_t *leaf_flag, int4 *tcell)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ncells) return;
    const double *bx = box + 4 * c.sys[i];
    const double h = ldexp(bx[3], -(c.level[i] + 1));
    half[i] = h;
    centre[3 * i] = __dadd_rn(bx[0], __dmul_rn((double)(2 * c.cx[i] + 1), h));
    centre[3 * i + 1] = __dadd_rn(bx[1], __dmul_rn((double)(2 * c.cy[i] + 1), h));
    centre[3 * i + 2] = __dadd_rn(bx[2], __dmul_rn((double)(2 * c.cz[i] + 1), h));
    leaf_flag[i] = c.nchild[i] == 0;
    tcell[i] = make_int4(c.cx[i] | c.level[i] << kLevels, c.cy[i] | c.nchild[i] << kLevels, c.cz[i],
                         c.child[i]);
}

// leaves[0, nleaves): the leaves in index order; leaves[nleaves, ncells): the
// cells with children in index (so breadth-first) order, for the downward pass
__global__ void k_compact_leaves(const uint32_t *flag, const uint32_t *pos, int64_t ncells,
                                 int32_t *leaves)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ncells) return;
    if (flag[i]) leaves[pos[i]] = (int32_t)i;
    else leaves[pos[ncells] + (i - pos[i])] = (int32_t)i;
}

// ----------------------------------------------------------- traversal
// MAC of Eq. (13), exact: centres (2c+1) 2^(21-l) and radii 2^(21-l) in units
// of the finest half-cell; (rA + rB)^2 < (theta*theta) |dc|^2.  The cells come
// as the packed records of k_cell_geometry.
constexpr int kCoordMask = (1 << kLevels) - 1;
__device__ __forceinline__ bool mac_accept(const int4 A, const int4 B, double theta2)
{
    const int la = A.x >> kLevels, lb = B.x >> kLevels;
    const long long ra = 1ll << (kLevels - la), rb = 1ll << (kLevels - lb);
    const long long dx = (2ll * (A.x & kCoordMask) + 1) * ra - (2ll * (B.x & kCoordMask) + 1) * rb;
    const long long dy = (2ll * (A.y & kCoordMask) + 1) * ra - (2ll * (B.y & kCoordMask) + 1) * rb;
    const long long dz = (2ll * A.z + 1) * ra - (2ll * B.z + 1) * rb;
    const long long d2 = dx * dx + dy * dy + dz * dz;
    const double lhs = (double)((ra + rb) * (ra + rb));
    return lhs < __dmul_rn(theta2, (double)d2);
}

// Position of a pair inside its target's row: the lanes that emit a pair of
// the same list for the same target share one atomic on that row's count.
// All lanes of the warp call it; lanes with want == false get 0.
__device__ __forceinline__ unsigned row_slot(unsigned *rows, int a, bool want)
{
    const int lane = threadIdx.x & 31;
    const unsigned act = __ballot_sync(0xffffffffu, want);
    unsigned slot = 0;
    if (want) {
        const unsigned peers = __match_any_sync(act, a);
        const int leader = __ffs(peers) - 1;
        unsigned base = 0;
        if (lane == leader) base = atomicAdd(&rows[a], (unsigned)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        slot = base + __popc(peers & ((1u << lane) - 1u));
    }
    return slot;
}

// One round of the breadth-first dual traversal.  The rounds are launched
// back to back without the host: round r reads its frontier size from
// counters[kTravFront + r] and adds the next round's to the word after it.
// counters: 0 = m2l, 1 = p2p, kTravOverflow = a frontier exceeded front_cap
// (every later round then does nothing).  Outputs beyond a list's capacity
// are counted but not written; the host grows what overflowed and reruns
// the whole traversal.  Each emitted pair also takes the next position in
// its target's row (rows_m2l / rows_p2p count the pairs of every target),
// kept in slot_m2l / slot_p2p beside the pair, so that the lists can be laid
// out by target without a sort by target.
constexpr int kTravOverflow = 16, kTravFront = 32, kTravMaxRounds = 960;
// blocks of a traversal round: 8 resident blocks of 256 threads per SM
constexpr int kTravBlocksPerSM = 8;
constexpr int kTravWarps = 8;            // warps of a traversal block (256 threads)

__global__ void __launch_bounds__(256)
k_traverse_round(const int4 *__restrict__ tc, int round, double theta2, const int2 *front,
                 unsigned front_cap, int2 *m2l, uint32_t *slot_m2l, unsigned *rows_m2l, unsigned m2l_cap,
                 int2 *p2p, uint32_t *slot_p2p, unsigned *rows_p2p, unsigned p2p_cap, int2 *next,
                 unsigned *counters)
{
    // the frontier size and the overflow flag, read once per block so that the
    // whole block takes the same way (the loop below has block barriers)
    __shared__ unsigned s_nf, s_stop;
    if (threadIdx.x == 0) {
        s_nf = counters[kTravFront + round];
        s_stop = s_nf == 0 || counters[kTravOverflow] != 0u;
    }
    __syncthreads();
    const unsigned nf = s_nf;
    if (s_stop) return;
    if (nf > front_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&counters[kTravOverflow], 1u);
        return;
    }
    unsigned *next_count = &counters[kTravFront + round + 1];
    // per-warp totals and block bases of the reservation, two sets used in turn
    __shared__ unsigned s_wsum[2][3][kTravWarps], s_base[2][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int par = 0;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned base = blockIdx.x * blockDim.x; base < nf; base += stride) {
        const unsigned t = base + threadIdx.x;
        const bool valid = t < nf;
        int a = 0, b = 0, na = 0, nb = 0;
        int4 A = make_int4(0, 0, 0, 0), B = A;
        if (valid) {
            const int2 pr = front[t];
            a = pr.x; b = pr.y;
            A = __ldg(tc + a);
            B = a == b ? A : __ldg(tc + b);
            na = A.y >> kLevels; nb = B.y >> kLevels;
        }
        // classify: kind 0 = M2L, 1 = P2P, 2 = open a (all children against b,
        // or all child pairs for a self pair), 3 = open b
        int kind = -1;
        if (valid) {
            if (a == b) kind = na == 0 ? 1 : 2;
            else if (mac_accept(A, B, theta2)) kind = 0;
            else if (na == 0 && nb == 0) kind = 1;
            else if (na == 0) kind = 3;
            else if (nb == 0) kind = 2;
            else kind = (A.x >> kLevels) <= (B.x >> kLevels) ? 2 : 3;
        }
        const unsigned n_next = kind == 2 ? (a == b ? (unsigned)(na * na) : (unsigned)na)
                                          : (kind == 3 ? (unsigned)nb : 0u);
        // slots in the three outputs: one atomic per block and output (the
        // counters are shared by the whole grid), lanes in thread order
        const unsigned want[3] = {kind == 0 ? 1u : 0u, kind == 1 ? 1u : 0u, n_next};
        unsigned incl[3];
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            incl[l] = want[l];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, incl[l], o);
                if (lane >= o) incl[l] += y;
            }
        }
        unsigned (*wsum)[kTravWarps] = s_wsum[par];
        if (lane == 31) {
#pragma unroll
            for (int l = 0; l < 3; ++l) wsum[l][warp] = incl[l];
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            const int l = threadIdx.x;
            unsigned run = 0;
            for (int w = 0; w < kTravWarps; ++w) {
                const unsigned v = wsum[l][w];
                wsum[l][w] = run;
                run += v;
            }
            s_base[par][l] = run ? atomicAdd(l == 0 ? &counters[0] : (l == 1 ? &counters[1] : next_count), run) : 0u;
        }
        __syncthreads();
        const unsigned o_m2l = s_base[par][0] + wsum[0][warp] + incl[0] - want[0];
        const unsigned o_p2p = s_base[par][1] + wsum[1][warp] + incl[1] - want[1];
        const unsigned o_next = s_base[par][2] + wsum[2][warp] + incl[2] - want[2];
        par ^= 1;
        const unsigned r_m2l = row_slot(rows_m2l, a, kind == 0);
        const unsigned r_p2p = row_slot(rows_p2p, a, kind == 1);
        if (kind == 0) {
            if (o_m2l < m2l_cap) { m2l[o_m2l] = make_int2(a, b); slot_m2l[o_m2l] = r_m2l; }
        } else if (kind == 1) {
            if (o_p2p < p2p_cap) { p2p[o_p2p] = make_int2(a, b); slot_p2p[o_p2p] = r_p2p; }
        }
        // the next frontier: a self pair opens into up to 64 child pairs, far
        // more than other entries, so a warp holding one writes its lanes'
        // children together (entry q of the warp's run goes to the lane whose
        // range holds it); otherwise each lane writes its own
        const int fc = kind == 2 ? A.w : B.w;
        if (__any_sync(0xffffffffu, n_next > 16)) {
            const unsigned wtot = __shfl_sync(0xffffffffu, incl[2], 31);
            const unsigned wbase = o_next - (incl[2] - want[2]);
            for (unsigned q0 = 0; q0 < wtot; q0 += 32) {
                const unsigned q = q0 + lane;
                // owner: the first lane whose inclusive end exceeds q
                int lo = 0;
#pragma unroll
                for (int st = 16; st > 0; st >>= 1) {
                    const unsigned e = __shfl_sync(0xffffffffu, incl[2], lo + st - 1);
                    if (e <= q) lo += st;
                }
                const unsigned ex = __shfl_sync(0xffffffffu, incl[2] - want[2], lo);
                const int oa = __shfl_sync(0xffffffffu, a, lo), ob = __shfl_sync(0xffffffffu, b, lo);
                const int of = __shfl_sync(0xffffffffu, fc, lo), ok = __shfl_sync(0xffffffffu, kind, lo);
                const int on = __shfl_sync(0xffffffffu, na, lo);
                if (q < wtot && wbase + q < front_cap) {
                    const int k = (int)(q - ex);
                    int2 v;
                    if (ok == 3) v = make_int2(oa, of + k);
                    else if (oa == ob) v = make_int2(of + k / on, of + k % on);
                    else v = make_int2(of + k, ob);
                    next[wbase + q] = v;
                }
            }
        } else if (kind == 2 && a == b) {
            for (int i = 0; i < na; ++i)
                for (int j = 0; j < na; ++j) {
                    const unsigned k = o_next + (unsigned)(i * na + j);
                    if (k < front_cap) next[k] = make_int2(fc + i, fc + j);
                }
        } else if (kind == 2) {
            for (int i = 0; i < na; ++i)
                if (o_next + i < front_cap) next[o_next + i] = make_int2(fc + i, b);
        } else if (kind == 3) {
            for (int j = 0; j < nb; ++j)
                if (o_next + j < front_cap) next[o_next + j] = make_int2(a, fc + j);
        }
    }
}

// ------------------------------------------------- lists laid out by target
// A pair goes to its row at the position the traversal gave it.
__global__ void k_list_scatter(const int2 *pairs, const uint32_t *slot, int64_t np,
                               const uint32_t *off, int32_t *src)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= np) return;
    const int2 p = pairs[k];
    src[off[p.x] + slot[k]] = p.y;
}

// Rows of a list sorted by source, in place, so that every build gives the
// same lists in the same order whatever order the traversal's atomics took.
// One warp per row: up to 32 entries in registers, up to kRowWarpMax in the
// warp's slice of shared memory (bitonic network, padded with ~0); longer rows
// are queued for k_row_sort_long.  With COUNT, the P2P interactions of every
// pair (targets x sources) are summed into *inter.
constexpr int kRowWarpMax = 1024, kRowBlockMax = 8192;

__device__ __forceinline__ void bitonic_smem(uint32_t *v, int n, int tid, int nthreads, bool warp)
{
    for (int k = 2; k <= n; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < (n >> 1); i += nthreads) {
                const int lo = 2 * i - (i & (j - 1)), hi = lo + j;
                const bool up = (lo & k) == 0;
                const uint32_t x = v[lo], y = v[hi];
                if ((x > y) == up) { v[lo] = y; v[hi] = x; }
            }
            if (warp) __syncwarp(); else __syncthreads();
        }
}

template <bool COUNT>
__global__ void __launch_bounds__(256)
k_row_sort(const uint32_t *off, int32_t *src, int64_t nrows, const int32_t *cbeg, const int32_t *cend,
           unsigned long long *inter, uint32_t *long_rows, unsigned *n_long, int warp_max)
{
    __shared__ uint32_t buf[8][kRowWarpMax];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * 8;
    unsigned long long acc = 0;
    for (int64_t r = blockIdx.x * 8ll + w; r < nrows; r += nwarps) {
        const uint32_t b0 = off[r], L = off[r + 1] - b0;
        if (L == 0) continue;
        if (COUNT) {
            unsigned long long s = 0;
            for (uint32_t k = lane; k < L; k += 32) {
                const int j = src[b0 + k];
                s += (unsigned long long)(cend[j] - cbeg[j]);
            }
            acc += s * (unsigned long long)(cend[r] - cbeg[r]);
        }
        if (L == 1) continue;
        if (L > (uint32_t)warp_max) {
            if (lane == 0) long_rows[atomicAdd(n_long, 1u)] = (uint32_t)r;
        } else if (L <= 32) {
            uint32_t v = lane < (int)L ? (uint32_t)src[b0 + lane] : ~0u;
#pragma unroll
            for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
                for (int j = k >> 1; j > 0; j >>= 1) {
                    const uint32_t o = __shfl_xor_sync(0xffffffffu, v, j);
                    const bool up = (lane & k) == 0, lower = (lane & j) == 0;
                    v = (lower == up) ? min(v, o) : max(v, o);
                }
            if (lane < (int)L) src[b0 + lane] = (int32_t)v;
        } else {
            int n = 64;
            while (n < (int)L) n <<= 1;
            uint32_t *v = buf[w];
            for (int k = lane; k < n; k += 32) v[k] = k < (int)L ? (uint32_t)src[b0 + k] : ~0u;
            __syncwarp();
            bitonic_smem(v, n, lane, 32, true);
            for (int k = lane; k < (int)L; k += 32) src[b0 + k] = (int32_t)v[k];
            __syncwarp();
        }
    }
    if (COUNT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0 && acc) atomicAdd(inter, acc);
    }
}

// The queued long rows, one block each; a row longer than block_max (at most
// kRowBlockMax) sets kErrLongRow in *err and is left for the host, which
// then sorts the whole list by (target, source) with the radix sort.
__global__ void __launch_bounds__(1024)
k_row_sort_long(const uint32_t *off, int32_t *src, const uint32_t *long_rows, const unsigned *n_long,
                int *err, int block_max)
{
    __shared__ uint32_t v[kRowBlockMax];
    const unsigned nl = *n_long;
    for (unsigned q = blockIdx.x; q < nl; q += gridDim.x) {
        const uint32_t r = long_rows[q], b0 = off[r], L = off[r + 1] - b0;
        if (L > (uint32_t)block_max) {
            if (threadIdx.x == 0) atomicOr(err, kErrLongRow);
            continue;
        }
        int n = 64;
        while (n < (int)L) n <<= 1;
        for (int k = threadIdx.x; k < n; k += blockDim.x) v[k] = k < (int)L ? (uint32_t)src[b0 + k] : ~0u;
        __syncthreads();
        bitonic_smem(v, n, threadIdx.x, blockDim.x, false);
        for (int k = threadIdx.x; k < (int)L; k += blockDim.x) src[b0 + k] = (int32_t)v[k];
        __syncthreads();
    }
}

__global__ void k_pack_pairs(const int2 *pairs, int64_t np, int cbits, uint64_t *keys,
                             uint32_t *vals)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= np) return;
    keys[k] = ((uint64_t)(uint32_t)pairs[k].x << cbits) | (uint32_t)pairs[k].y;
    vals[k] = (uint32_t)k;
}

// CSR offsets: off[c] = first sorted pair whose target is >= c.
__global__ void k_row_offsets(const uint64_t *keys, int64_t np, int cbits, int64_t ncells,
                              int32_t *off)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c > ncells) return;
    int64_t L = 0, R = np;
    while (L < R) {
        int64_t mid = (L + R) >> 1;
        if ((int64_t)(keys[mid] >> cbits) < c) L = mid + 1; else R = mid;
    }
    off[c] = (int32_t)L;
}

__global__ void k_unpack_src(const uint64_t *keys, int64_t np, int cbits, int32_t *src)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < np) src[k] = (int32_t)(keys[k] & ((1ull << cbits) - 1ull));
}

__global__ void k_p2p_interactions(const uint64_t *keys, int64_t np, int cbits, CellArrays c,
                                   unsigned long long *total)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (k < np) {
        const int a = (int)(keys[k] >> cbits), b = (int)(keys[k] & ((1ull << cbits) - 1ull));
        v = (unsigned long long)(c.end[a] - c.begin[a]) * (unsigned long long)(c.end[b] - c.begin[b]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, v);
}

// --------------------------------------------------- D-table offset keys
// key = level gap (5 bits) | target-is-finer (1 bit) | three 17-bit biased
// offsets v in units of the finer cell's half side u.  D rows are stored for
// the unit-free offset v; a pair's real offset is u v with u = side / 2^(lf+1)
// a power of two, so one row serves every level and every system.
__device__ __forceinline__ uint64_t hash64(uint64_t x)
{
    x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

// Offset keys of the M2L pairs, one warp per target row (CSR order): the
// key of a pair is its level gap, which side is finer and the centre offset
// in finer half-cells; equal keys share one derivative row.
__global__ void k_offset_keys(CellArrays c, const int32_t *off, const int32_t *src, int64_t nrows,
                              unsigned long long *table, uint32_t hmask, uint32_t *slot_of,
                              int *err, unsigned *max_gap)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; a < nrows; a += nwarps) {
        const int k0 = off[a], k1 = off[a + 1];
        if (k0 == k1) continue;
        const int la = c.level[a];
        const long long ax = 2ll * c.cx[a] + 1, ay = 2ll * c.cy[a] + 1, az = 2ll * c.cz[a] + 1;
        unsigned gmax = 0;
        for (int k = k0 + lane; k < k1; k += 32) {
            const int b = src[k];
            const int lb = c.level[b], lf = la > lb ? la : lb;
            const long long sa = 1ll << (lf - la), sb = 1ll << (lf - lb);
            long long d[3] = {ax * sa - (2ll * c.cx[b] + 1) * sb, ay * sa - (2ll * c.cy[b] + 1) * sb,
                              az * sa - (2ll * c.cz[b] + 1) * sb};
            const int gap = la > lb ? la - lb : lb - la;
            gmax = gap > (int)gmax ? (unsigned)gap : gmax;
            uint64_t key = (uint64_t)gap << 52 | (uint64_t)(la > lb) << 51;
            bool bad = false;
            for (int i = 0; i < 3; ++i) {
                if (d[i] < -kKeyBias || d[i] >= kKeyBias) { bad = true; break; }
                key |= (uint64_t)(d[i] + kKeyBias) << (34 - 17 * i);
            }
            if (bad) { atomicOr(err, kErrKeyRange); slot_of[k] = 0; continue; }
            uint32_t h = (uint32_t)hash64(key) & hmask;
            bool placed = false;
            for (uint32_t probe = 0; probe <= hmask; ++probe) {
                unsigned long long cur = table[h];
                if (cur == key) { placed = true; break; }
                if (cur == ~0ull) {
                    unsigned long long prev = atomicCAS(&table[h], ~0ull, (unsigned long long)key);
                    if (prev == ~0ull || prev == key) { placed = true; break; }
                }
                h = (h + 1) & hmask;
            }
            if (!placed) { atomicOr(err, kErrHashFull); h = 0; }
            slot_of[k] = h;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gmax = max(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
        if (lane == 0 && gmax) atomicMax(max_gap, gmax);
    }
}

__global__ void k_slot_flags(const unsigned long long *table, uint32_t H, uint32_t *flag)
{
    uint32_t h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h < H) flag[h] = table[h] != ~0ull;
}

__global__ void k_slot_compact(const unsigned long long *table, uint32_t H, const uint32_t *dense,
                               uint64_t *dkeys)
{
    uint32_t h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h < H && table[h] != ~0ull) dkeys[dense[h]] = table[h];
}

// Which colliding key wins a hash slot depends on timing, so slot order is
// not reproducible: the distinct keys are sorted by value and a pair's D row
// is the rank of its key (rank_of[dense index]).
__global__ void k_slot_to_dense(int32_t *didx, int64_t np, const uint32_t *dense, const uint32_t *rank_of)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < np) didx[k] = (int32_t)rank_of[dense[(uint32_t)didx[k]]];
}

__global__ void k_iota(uint32_t *v, int64_t n)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) v[k] = (uint32_t)k;
}

// Distinct keys (n <= kRankSmall) sorted in place in one block: a key's rank
// is the number of smaller keys.  The result equals the radix sort's.
constexpr int kRankSmall = 4096;

__global__ void __launch_bounds__(1024) k_rank_small(uint64_t *keys, int n, uint32_t *rank_of)
{
    extern __shared__ uint64_t sk[];
    for (int i = threadIdx.x; i < n; i += blockDim.x) sk[i] = keys[i];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const uint64_t v = sk[i];
        int r = 0;
        for (int j = 0; j < n; ++j) r += sk[j] < v;
        rank_of[i] = (uint32_t)r;
        keys[r] = v;                 // every read is from shared memory
    }
}

__global__ void k_rank_of(const uint32_t *old_of_rank, int64_t n, uint32_t *rank_of)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) rank_of[old_of_rank[r]] = (uint32_t)r;
}

inline unsigned grid(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

CellArrays cells_of(fmm_tree *t)
{
    CellArrays c;
    c.level = (int32_t *)t->b_level.ptr; c.parent = (int32_t *)t->b_parent.ptr;
    c.child = (int32_t *)t->b_child.ptr; c.nchild = (int32_t *)t->b_nchild.ptr;
    c.begin = (int32_t *)t->b_begin.ptr; c.end = (int32_t *)t->b_end.ptr;
    c.cx = (int32_t *)t->b_cx.ptr; c.cy = (int32_t *)t->b_cy.ptr; c.cz = (int32_t *)t->b_cz.ptr;
    c.sys = (int32_t *)t->b_sys.ptr;
    return c;
}

// Grow a buffer, keeping its first keep_bytes.
fmm_status grow_keep(fmm_tree *t, DevBuf &b, size_t bytes, size_t keep_bytes)
{
    if (b.bytes >= bytes) return FMM_OK;
    DevBuf nb;
    size_t want = std::max(bytes, b.bytes + b.bytes / 2);
    FMM_TRY(ensure(t, nb, want));
    if (keep_bytes && b.ptr)
        FMM_TRY(cuda_check(t, cudaMemcpyAsync(nb.ptr, b.ptr, keep_bytes, cudaMemcpyDeviceToDevice,
                                              t->stream), "grow copy"));
    release(t, b);
    b = nb;
    return FMM_OK;
}

fmm_status read_err(fmm_tree *t)
{
    int e = 0;
    FMM_TRY(cuda_check(t, cudaMemcpyAsync(&e, t->b_err.ptr, sizeof(int), cudaMemcpyDeviceToHost,
                                          t->stream), "read error word"));
    FMM_TRY(cuda_check(t, cudaStreamSynchronize(t->stream), "sync"));
    if (e & kErrNonFinite) { t->err = "non-finite particle position"; return FMM_EINVAL; }
    if (e & kErrKeyRange) {
        t->err = "an accepted M2L offset exceeds 2^16 finer half-cells (theta too small for the tree)";
        return FMM_EINVAL;
    }
    if (e & kErrSortWait) { t->err = "a bounded wait of the radix sort gave up"; return FMM_ETIMEOUT; }
    return FMM_OK;
}

void record(fmm_tree *t, int i)
{
    if (t->profiling) cudaEventRecord(t->ev[i], t->stream);
}

}  // namespace

// ---------------------------------------------------------------------------
// keys of one system, with the digit counts of their radix sort (hist: the
// sort's scratch, its head zeroed here)
static void morton_keys(cudaStream_t st, const double *pos, int64_t n, uint64_t *keys,
                        uint32_t *idx, unsigned long long *box_scratch, double *box_out, int *err,
                        uint32_t *hist, int64_t *launches)
{
    k_box_init<<<1, 32, 0, st>>>(box_scratch);
    k_bbox<<<(unsigned)std::min<int64_t>(grid(n, 256), 4 * (int64_t)sm_count()), 256, 0, st>>>(pos, n, box_scratch, err);
    k_box_final<<<1, 1, 0, st>>>(box_scratch, box_out);
    cudaMemsetAsync(hist, 0, 4 * (size_t)kRadixHead, st);
    const int64_t ntiles = (n + kRadixTile - 1) / kRadixTile;
    k_keys<<<(unsigned)std::min<int64_t>(grid(n, 256), 4 * (int64_t)sm_count()), 256, 0, st>>>(
        pos, n, box_out, keys, idx, hist, (uint64_t *)(hist + kRadixHead), ntiles * 256);
    *launches += 4;
}

void morton_order_prepare()
{
    cudaFuncAttributes fa;
    const void *kerns[] = {(const void *)k_box_init, (const void *)k_bbox, (const void *)k_box_final,
                           (const void *)k_keys};
    for (const void *k : kerns)
        if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) cudaGetLastError();
    radix_sort_prepare();
}

fmm_status morton_order_raw(cudaStream_t st, const double *pos, int64_t n, uint64_t *keys,
                            uint32_t *idx, uint64_t *keys2, uint32_t *idx2, uint32_t *hist,
                            unsigned long long *box_scratch, double *box_out, int *err,
                            int64_t *launches)
{
    morton_keys(st, pos, n, keys, idx, box_scratch, box_out, err, hist, launches);
    radix_sort_pairs(keys, idx, keys2, idx2, n, 3 * kLevels, hist, err, st, launches, true);
    return FMM_OK;
}

fmm_status build_tree(fmm_tree *t, const double *pos, const double *mom)
{
    const int64_t n = t->n;
    const int nsys = (int)t->sys_off.size() - 1;
    cudaStream_t st = t->stream;
    t->have_lists = false;
    t->ncells = t->nleaves = 0;
    t->nlevels = 0;
    t->level_begin.clear();
    if (n == 0) return FMM_OK;

    FMM_TRY(ensure(t, t->b_keys, 8 * n));
    FMM_TRY(ensure(t, t->b_keys2, 8 * n));
    FMM_TRY(ensure(t, t->b_idx, 4 * n));
    FMM_TRY(ensure(t, t->b_idx2, 4 * n));
    FMM_TRY(ensure(t, t->b_hist, radix_hist_bytes(n)));
    FMM_TRY(ensure(t, t->b_scan_tmp, scan_scratch_bytes(std::max<int64_t>(n, 1 << 20) * 8)));
    FMM_TRY(ensure(t, t->b_px, 8 * n));
    FMM_TRY(ensure(t, t->b_py, 8 * n));
    FMM_TRY(ensure(t, t->b_pz, 8 * n));
    FMM_TRY(ensure(t, t->b_S, 8 * n * t->nS));
    FMM_TRY(ensure(t, t->b_perm, 4 * n));
    FMM_TRY(ensure(t, t->b_sysoff, 8 * (size_t)(nsys + 1)));
    FMM_TRY(ensure(t, t->b_sysbox, 32 * (size_t)nsys + 48 * (size_t)nsys));
    uint64_t *keys = (uint64_t *)t->b_keys.ptr;
    uint32_t *idx = (uint32_t *)t->b_idx.ptr;
    int64_t *off = (int64_t *)t->b_sysoff.ptr;
    double *sbox = (double *)t->b_sysbox.ptr;                               // [nsys][4]
    unsigned long long *sbox_raw = (unsigned long long *)(sbox + 4 * nsys); // [nsys][6]

    record(t, 0);
    cudaMemsetAsync(t->b_err.ptr, 0, sizeof(int), st);
    FMM_TRY(cuda_check(t, cudaMemcpyAsync(off, t->sys_off.data(), 8 * (size_t)(nsys + 1),
                                          cudaMemcpyHostToDevice, st), "system offsets"));
    if (nsys == 1) {
        morton_keys(st, pos, n, keys, idx, sbox_raw, sbox, (int *)t->b_err.ptr, (uint32_t *)t->b_hist.ptr,
                    &t->launches);
    } else {
        // particle -> system (kept in b_idx2 until the sort needs it)
        FMM_TRY(ensure(t, t->b_lval2, 4 * n));
        int32_t *sys_of = (int32_t *)t->b_lval2.ptr;
        k_sys_of<<<grid(n, 256), 256, 0, st>>>(off, nsys, n, sys_of);
        k_box_init_seg<<<grid(6 * nsys, 256), 256, 0, st>>>(sbox_raw, nsys);
        k_bbox_seg<<<grid(n, 256), 256, 0, st>>>(pos, n, sys_of, sbox_raw, (int *)t->b_err.ptr);
        k_box_final_seg<<<grid(nsys, 128), 128, 0, st>>>(sbox_raw, nsys, sbox);
        k_keys_seg<<<grid(n, 256), 256, 0, st>>>(pos, n, sys_of, sbox, keys, idx);
        t->launches += 5;
    }
    record(t, 1);
    radix_sort_pairs(keys, idx, (uint64_t *)t->b_keys2.ptr, (uint32_t *)t->b_idx2.ptr, n,
                     3 * kLevels, (uint32_t *)t->b_hist.ptr, (int *)t->b_err.ptr, st, &t->launches,
                     nsys == 1);                   // one system: k_keys counted the digits
    if (nsys > 1) {
        // stable second pass by system: order = (system, key, original index)
        FMM_TRY(ensure(t, t->b_lkeys, 8 * n));
        FMM_TRY(ensure(t, t->b_lkeys2, 8 * n));
        uint64_t *skeys = (uint64_t *)t->b_lkeys.ptr, *key_of = (uint64_t *)t->b_lkeys2.ptr;
        k_sys_keys<<<grid(n, 256), 256, 0, st>>>(keys, idx, (const int32_t *)t->b_lval2.ptr, n,
                                                 skeys, key_of);
        int sbits = 1;
        while ((1 << sbits) < nsys) ++sbits;
        radix_sort_pairs(skeys, idx, (uint64_t *)t->b_keys2.ptr, (uint32_t *)t->b_idx2.ptr, n,
                         sbits, (uint32_t *)t->b_hist.ptr, (int *)t->b_err.ptr, st, &t->launches);
        k_regather_keys<<<grid(n, 256), 256, 0, st>>>(key_of, idx, n, keys);
        t->launches += 2;
    }
    k_gather<<<grid(n, 256), 256, 0, st>>>(pos, mom, t->nS, idx, n, (double *)t->b_px.ptr,
                                           (double *)t->b_py.ptr, (double *)t->b_pz.ptr,
                                           (double *)t->b_S.ptr, (int32_t *)t->b_perm.ptr);
    ++t->launches;
    record(t, 2);

    // ---- cells, level by level on the device (level 0 holds one root per system);
    // the host reads the level counts once per batch of levels
    FMM_TRY(ensure(t, t->b_ctl, 4 * kCtlWords));
    unsigned *ctl = (unsigned *)t->b_ctl.ptr;
    DevBuf *cb[10] = {&t->b_level, &t->b_parent, &t->b_child, &t->b_nchild, &t->b_begin,
                      &t->b_end, &t->b_cx, &t->b_cy, &t->b_cz, &t->b_sys};
    int64_t cap = std::max<int64_t>(t->b_level.bytes / 4,
                                    std::max<int64_t>(1024, 5 * (n / std::max(1, t->max_leaf)) + 64 + 2 * nsys));
    const unsigned lgrid = (unsigned)(8 * sm_count());
    std::vector<unsigned> hc(kCtlWords);
    int nlev = 0;
    for (;;) {
        for (DevBuf *b : cb) FMM_TRY(ensure(t, *b, 4 * cap));
        FMM_TRY(ensure(t, t->b_flags, 4 * cap));
        FMM_TRY(ensure(t, t->b_scan, 4 * cap));
        FMM_TRY(ensure(t, t->b_front, 8 * 8 * cap));      // child begin/end of every octant
        CellArrays c = cells_of(t);
        uint32_t *cnt = (uint32_t *)t->b_flags.ptr, *off8 = (uint32_t *)t->b_scan.ptr;
        int32_t *cbeg = (int32_t *)t->b_front.ptr, *cend = cbeg + 8 * cap;
        k_roots<<<grid(nsys, 128), 128, 0, st>>>(c, off, nsys);
        k_level_init<<<1, kCtlWords, 0, st>>>(ctl, nsys);
        t->launches += 2;
        int level = 0;
        bool overflow = false;
        for (;;) {
            const int end = std::min(level + kLevelBatch, kLevels + 1);
            for (; level < end; ++level) {
                k_level_ranges<<<lgrid, 256, 0, st>>>(c, ctl, level, t->max_leaf, keys, cbeg, cend, cnt);
                k_level_scan<<<1, 1024, 0, st>>>(ctl, level, cnt, off8, cap);
                k_level_write<<<lgrid, 256, 0, st>>>(c, ctl, level, cbeg, cend, off8);
                t->launches += 3;
            }
            FMM_TRY(cuda_check(t, cudaMemcpyAsync(hc.data(), ctl, 4 * kCtlWords, cudaMemcpyDeviceToHost, st),
                               "level counts"));
            FMM_TRY(cuda_check(t, cudaStreamSynchronize(st), "sync"));
            if (hc[kCtlOverflow]) {
                overflow = true;
                break;
            }
            // done once a level came out empty (or the deepest level was processed)
            if (hc[kCtlLevel + level + 1] == hc[kCtlLevel + level] || level > kLevels) break;
        }
        if (!overflow) {
            // levels 0 .. nlev - 1 hold cells
            nlev = 1;
            while (nlev <= kLevels && hc[kCtlLevel + nlev + 1] > hc[kCtlLevel + nlev]) ++nlev;
            break;
        }
        cap *= 2;
    }
    t->level_begin.assign(hc.begin() + kCtlLevel, hc.begin() + kCtlLevel + nlev + 1);
    t->ncells = t->level_begin.back();
    t->nlevels = nlev;
    CellArrays c = cells_of(t);
    const int64_t nc = t->ncells;
    FMM_TRY(ensure(t, t->b_centre, 8 * 3 * nc));
    FMM_TRY(ensure(t, t->b_half, 8 * nc));
    FMM_TRY(ensure(t, t->b_flags, 4 * (nc + 1)));
    FMM_TRY(ensure(t, t->b_scan, 4 * (nc + 1)));
    uint32_t *flags = (uint32_t *)t->b_flags.ptr, *posc = (uint32_t *)t->b_scan.ptr;
    cudaMemsetAsync(flags + nc, 0, 4, st);
    FMM_TRY(ensure(t, t->b_tcell, 16 * nc));
    k_cell_geometry<<<grid(nc, 256), 256, 0, st>>>(c, nc, sbox, (double *)t->b_centre.ptr,
                                                    (double *)t->b_half.ptr, flags, (int4 *)t->b_tcell.ptr);
    exclusive_scan_u32(flags, posc, nc + 1, (uint32_t *)t->b_scan_tmp.ptr, st, &t->launches);
    uint32_t nleaves = 0;
    FMM_TRY(cuda_check(t, cudaMemcpyAsync(&nleaves, posc + nc, 4, cudaMemcpyDeviceToHost, st),
                       "leaf count"));
    FMM_TRY(ensure(t, t->b_leaves, 4 * (size_t)nc));
    k_compact_leaves<<<grid(nc, 256), 256, 0, st>>>(flags, posc, nc, (int32_t *)t->b_leaves.ptr);
    t->launches += 2;
    t->sys_box.assign(4 * (size_t)nsys, 0.0);
    FMM_TRY(cuda_check(t, cudaMemcpyAsync(t->sys_box.data(), sbox, 32 * (size_t)nsys,
                                          cudaMemcpyDeviceToHost, st), "box"));
    record(t, 3);
    FMM_TRY(read_err(t));
    t->nleaves = nleaves;
    t->lo[0] = t->sys_box[0]; t->lo[1] = t->sys_box[1]; t->lo[2] = t->sys_box[2];
    t->side = t->sys_box[3];
    std::vector<int> es((size_t)nsys);
    for (int s = 0; s < nsys; ++s) es[s] = std::ilogb(t->sys_box[4 * s + 3]);
    FMM_TRY(ensure(t, t->b_syseside, 4 * (size_t)nsys));
    FMM_TRY(cuda_check(t, cudaMemcpyAsync(t->b_syseside.ptr, es.data(), 4 * (size_t)nsys,
                                          cudaMemcpyHostToDevice, st), "system sides"));
    FMM_TRY(cuda_check(t, cudaStreamSynchronize(st), "sync"));
    return FMM_OK;
}

fmm_status build_lists(fmm_tree *t, double theta)
{
    cudaStream_t st = t->stream;
    t->have_lists = false;
    t->tc_plan = false;
    t->sym_plan = false;
    t->n_m2l = t->n_p2p = t->n_p2p_inter = t->n_doff = 0;
    t->d_p = -1;
    if (t->n == 0) { t->theta = theta; t->have_lists = true; return FMM_OK; }
    const int64_t nc = t->ncells;
    CellArrays c = cells_of(t);
    const double theta2 = theta * theta;

    // ---- breadth-first dual traversal: a pair's two levels add up to at
    // least its round, so 2 * nlevels rounds empty the frontier; they run as
    // one batch of launches with one host sync (more batches if not)
    FMM_TRY(ensure(t, t->b_counters, 4 * (kTravFront + kTravMaxRounds + 64)));
    unsigned *cnt = (unsigned *)t->b_counters.ptr;
    // row counts of both lists: [0, nc] M2L, [nc + 1, 2 nc + 1] P2P (the last
    // word of each stays 0 and becomes the total under the exclusive scan)
    FMM_TRY(ensure(t, t->b_rows, 8 * (size_t)(nc + 1)));
    unsigned *rows = (unsigned *)t->b_rows.ptr;
    const int nsys = (int)t->sys_off.size() - 1;
    size_t m2l_cap = std::max<size_t>(4096, t->m2l_cap_hint), p2p_cap = std::max<size_t>(4096, 40 * (size_t)t->nleaves);
    size_t front_cap = std::max<size_t>({(size_t)4096, (size_t)nsys, 16 * (size_t)t->nleaves,
                                         t->b_front.bytes / 8, t->b_front2.bytes / 8});
    std::vector<unsigned> hc((size_t)kTravFront + kTravMaxRounds + 1);
    const int batch = 2 * std::max(t->nlevels, 1) + 1;
    for (;;) {
        FMM_TRY(grow_keep(t, t->b_m2l_raw, 8 * m2l_cap, 0));
        FMM_TRY(grow_keep(t, t->b_p2p_raw, 8 * p2p_cap, 0));
        FMM_TRY(grow_keep(t, t->b_m2l_slot, 4 * (t->b_m2l_raw.bytes / 8), 0));
        FMM_TRY(grow_keep(t, t->b_p2p_slot, 4 * (t->b_p2p_raw.bytes / 8), 0));
        FMM_TRY(grow_keep(t, t->b_front, 8 * front_cap, 0));
        FMM_TRY(grow_keep(t, t->b_front2, 8 * front_cap, 0));
        m2l_cap = t->b_m2l_raw.bytes / 8;
        p2p_cap = t->b_p2p_raw.bytes / 8;
        front_cap = std::min(t->b_front.bytes, t->b_front2.bytes) / 8;
        int2 *fr[2] = {(int2 *)t->b_front.ptr, (int2 *)t->b_front2.ptr};
        FMM_TRY(cuda_check(t, cudaMemsetAsync(cnt, 0, 4 * (kTravFront + kTravMaxRounds + 1), st),
                           "counters"));
        FMM_TRY(cuda_check(t, cudaMemsetAsync(rows, 0, 8 * (size_t)(nc + 1), st), "row counts"));
        k_root_pairs<<<grid(nsys, 128), 128, 0, st>>>(fr[0], nsys, cnt + kTravFront);
        ++t->launches;
        int r = 0;
        bool retry = false;
        const unsigned trav_blocks = (unsigned)(kTravBlocksPerSM * sm_count());
        for (;;) {
            const int end = std::min(r + batch, kTravMaxRounds);
            for (; r < end; ++r) {
                k_traverse_round<<<trav_blocks, 256, 0, st>>>(
                    (const int4 *)t->b_tcell.ptr, r, theta2, fr[r & 1], (unsigned)front_cap,
                    (int2 *)t->b_m2l_raw.ptr, (uint32_t *)t->b_m2l_slot.ptr, rows, (unsigned)m2l_cap,
                    (int2 *)t->b_p2p_raw.ptr, (uint32_t *)t->b_p2p_slot.ptr, rows + nc + 1,
                    (unsigned)p2p_cap, fr[(r + 1) & 1], cnt);
                ++t->launches;
            }
            FMM_TRY(cuda_check(t, cudaMemcpyAsync(hc.data(), cnt, 4 * (size_t)(kTravFront + r + 1),
                                                  cudaMemcpyDeviceToHost, st), "counters"));
            FMM_TRY(cuda_check(t, cudaStreamSynchronize(st), "sync"));
            unsigned fmax = 0;
            for (int k = 0; k <= r; ++k) fmax = std::max(fmax, hc[kTravFront + k]);
            if (hc[kTravOverflow] || fmax > front_cap) {
                front_cap = std::max<size_t>(2 * front_cap, 2 * (size_t)fmax);
                retry = true;
            }
            if (hc[0] > m2l_cap) { m2l_cap = 2 * (size_t)hc[0]; retry = true; }
            if (hc[1] > p2p_cap) { p2p_cap = 2 * (size_t)hc[1]; retry = true; }
            if (retry || hc[kTravFront + r] == 0) break;
            if (r >= kTravMaxRounds) {
                t->err = "the dual traversal did not end within its round limit";
                return FMM_EINVAL;
            }
        }
        if (!retry) break;
    }
    const unsigned host_cnt[2] = {hc[0], hc[1]};
    const int64_t nm2l = host_cnt[0], np2p = host_cnt[1];
    t->m2l_cap_hint = (size_t)nm2l + nm2l / 8;

    // ---- both lists laid out by target (CSR).  Normally: offsets from the
    // row counts of the traversal, each pair to the position it was given,
    // rows sorted by source.  A row too long for the row sort (flag in
    // counter word 6, seen at the next host sync) sends both lists through
    // the radix sort of (target, source) keys instead; both give the same
    // lists.  The sorts report a wait that gave up in counter word 14.
    FMM_TRY(ensure(t, t->b_scan_tmp, scan_scratch_bytes(std::max<int64_t>(nc + 1, 1 << 20) * 8)));
    FMM_TRY(ensure(t, t->b_m2l_src, 4 * std::max<int64_t>(nm2l, 1)));
    FMM_TRY(ensure(t, t->b_m2l_didx, 4 * std::max<int64_t>(nm2l, 1)));
    FMM_TRY(ensure(t, t->b_m2l_off, 4 * (nc + 1)));
    FMM_TRY(ensure(t, t->b_p2p_src, 4 * std::max<int64_t>(np2p, 1)));
    FMM_TRY(ensure(t, t->b_p2p_off, 4 * (nc + 1)));
    FMM_TRY(ensure(t, t->b_long, 8 * (size_t)(nc + 1)));
    int *sort_err = (int *)(cnt + 14), *long_err = (int *)(cnt + 6);
    unsigned *n_long = cnt + 4;                          // queued long rows: M2L, P2P
    unsigned long long *inter_d = (unsigned long long *)(cnt + 8);
    int32_t *m2l_off = (int32_t *)t->b_m2l_off.ptr, *p2p_off = (int32_t *)t->b_p2p_off.ptr;
    int32_t *m2l_src = (int32_t *)t->b_m2l_src.ptr, *p2p_src = (int32_t *)t->b_p2p_src.ptr;
    int cbits = 1;
    while ((1ll << cbits) < nc) ++cbits;
    // FMM_ROW_SORT_LIMIT (tests) lowers the longest row the row sorts take
    int row_lim = kRowBlockMax;
    if (const char *env = getenv("FMM_ROW_SORT_LIMIT")) row_lim = std::min(std::max(2, atoi(env)), kRowBlockMax);
    auto layout_rows = [&]() {
        cudaMemsetAsync(cnt + 4, 0, 4 * 6, st);          // words 4 .. 9: long rows, flag, P2P count
        exclusive_scan_u32(rows, (uint32_t *)m2l_off, nc + 1, (uint32_t *)t->b_scan_tmp.ptr, st, &t->launches);
        exclusive_scan_u32(rows + nc + 1, (uint32_t *)p2p_off, nc + 1, (uint32_t *)t->b_scan_tmp.ptr, st,
                           &t->launches);
        uint32_t *lq = (uint32_t *)t->b_long.ptr;
        const unsigned rgrid = (unsigned)std::min<int64_t>((nc + 7) / 8, 6 * (int64_t)sm_count());
        if (nm2l > 0)
            k_list_scatter<<<grid(nm2l, 256), 256, 0, st>>>((const int2 *)t->b_m2l_raw.ptr,
                                                            (const uint32_t *)t->b_m2l_slot.ptr, nm2l,
                                                            (const uint32_t *)m2l_off, m2l_src);
        if (np2p > 0)
            k_list_scatter<<<grid(np2p, 256), 256, 0, st>>>((const int2 *)t->b_p2p_raw.ptr,
                                                            (const uint32_t *)t->b_p2p_slot.ptr, np2p,
                                                            (const uint32_t *)p2p_off, p2p_src);
        k_row_sort<false><<<rgrid, 256, 0, st>>>((const uint32_t *)m2l_off, m2l_src, nc, c.begin, c.end,
                                                  nullptr, lq, n_long, std::min(row_lim, kRowWarpMax));
        k_row_sort<true><<<rgrid, 256, 0, st>>>((const uint32_t *)p2p_off, p2p_src, nc, c.begin, c.end,
                                                 inter_d, lq + nc + 1, n_long + 1,
                                                 std::min(row_lim, kRowWarpMax));
        k_row_sort_long<<<(unsigned)sm_count(), 1024, 0, st>>>((const uint32_t *)m2l_off, m2l_src, lq,
                                                                n_long, long_err, row_lim);
        k_row_sort_long<<<(unsigned)sm_count(), 1024, 0, st>>>((const uint32_t *)p2p_off, p2p_src,
                                                                lq + nc + 1, n_long + 1, long_err, row_lim);
        t->launches += 6;
    };
    auto layout_radix = [&]() -> fmm_status {
        const int64_t nmax = std::max<int64_t>({nm2l, np2p, 1});
        FMM_TRY(ensure(t, t->b_lkeys, 8 * nmax));
        FMM_TRY(ensure(t, t->b_lkeys2, 8 * nmax));
        FMM_TRY(ensure(t, t->b_lval, 4 * nmax));
        FMM_TRY(ensure(t, t->b_lval2, 4 * nmax));
        FMM_TRY(ensure(t, t->b_hist, radix_hist_bytes(nmax)));
        uint64_t *lk = (uint64_t *)t->b_lkeys.ptr, *lk2 = (uint64_t *)t->b_lkeys2.ptr;
        uint32_t *lv = (uint32_t *)t->b_lval.ptr, *lv2 = (uint32_t *)t->b_lval2.ptr;
        cudaMemsetAsync(cnt + 6, 0, 4 * 4, st);          // words 6 .. 9: flag, P2P count
        k_pack_pairs<<<grid(np2p, 256), 256, 0, st>>>((const int2 *)t->b_p2p_raw.ptr, np2p, cbits, lk, lv);
        radix_sort_pairs(lk, lv, lk2, lv2, np2p, 2 * cbits, (uint32_t *)t->b_hist.ptr, sort_err, st,
                         &t->launches);
        k_row_offsets<<<grid(nc + 1, 256), 256, 0, st>>>(lk, np2p, cbits, nc, p2p_off);
        k_unpack_src<<<grid(np2p, 256), 256, 0, st>>>(lk, np2p, cbits, p2p_src);
        k_p2p_interactions<<<grid(np2p, 256), 256, 0, st>>>(lk, np2p, cbits, c, inter_d);
        t->launches += 4;
        if (nm2l > 0) {
            k_pack_pairs<<<grid(nm2l, 256), 256, 0, st>>>((const int2 *)t->b_m2l_raw.ptr, nm2l, cbits, lk, lv);
            radix_sort_pairs(lk, lv, lk2, lv2, nm2l, 2 * cbits, (uint32_t *)t->b_hist.ptr, sort_err,
                             st, &t->launches);
            k_unpack_src<<<grid(nm2l, 256), 256, 0, st>>>(lk, nm2l, cbits, m2l_src);
            t->launches += 2;
        }
        k_row_offsets<<<grid(nc + 1, 256), 256, 0, st>>>(lk, nm2l, cbits, nc, m2l_off);
        ++t->launches;
        return FMM_OK;
    };
    cudaMemsetAsync(sort_err, 0, 4, st);
    layout_rows();

    // ---- distinct M2L offsets (rows of the derivative table).  One host sync
    // reads everything at once: the hash status, the long-row flag, the
    // distinct count, the largest level gap and the P2P interaction count;
    // a full hash table or a long row (rare) redoes the part concerned.
    int64_t ndoff = 0;
    int serr = 0, le = 0;
    unsigned long long inter = 0;
    bool dsort = false;                    // the distinct keys went through the radix sort
    if (nm2l > 0) {
        uint32_t H = 1u << 16;
        while (H < 4 * (uint32_t)std::min<int64_t>(nm2l, 1 << 22) && H < (1u << 20)) H <<= 1;
        uint32_t nd = 0;
        for (;;) {
            FMM_TRY(ensure(t, t->b_hash, 8 * (size_t)H));
            FMM_TRY(ensure(t, t->b_flags, 4 * ((size_t)H + 1)));
            FMM_TRY(ensure(t, t->b_scan, 4 * ((size_t)H + 1)));
            FMM_TRY(ensure(t, t->b_scan_tmp, scan_scratch_bytes((int64_t)H + 1)));
            cudaMemsetAsync(t->b_hash.ptr, 0xff, 8 * (size_t)H, st);
            cudaMemsetAsync(t->b_err.ptr, 0, sizeof(int), st);
            cudaMemsetAsync(cnt + 12, 0, 4, st);
            k_offset_keys<<<(unsigned)std::min<int64_t>((nc + 7) / 8, 8 * (int64_t)sm_count()), 256, 0, st>>>(
                c, m2l_off, m2l_src, nc, (unsigned long long *)t->b_hash.ptr, H - 1,
                (uint32_t *)t->b_m2l_didx.ptr, (int *)t->b_err.ptr, cnt + 12);
            uint32_t *flag = (uint32_t *)t->b_flags.ptr, *dense = (uint32_t *)t->b_scan.ptr;
            cudaMemsetAsync(flag + H, 0, 4, st);
            k_slot_flags<<<grid(H, 256), 256, 0, st>>>((unsigned long long *)t->b_hash.ptr, H, flag);
            exclusive_scan_u32(flag, dense, (int64_t)H + 1, (uint32_t *)t->b_scan_tmp.ptr, st, &t->launches);
            t->launches += 2;
            int e = 0;
            unsigned gmax = 0;
            FMM_TRY(cuda_check(t, cudaMemcpyAsync(&e, t->b_err.ptr, 4, cudaMemcpyDeviceToHost, st), "err"));
            FMM_TRY(cuda_check(t, cudaMemcpyAsync(&le, long_err, 4, cudaMemcpyDeviceToHost, st), "rows"));
            FMM_TRY(cuda_check(t, cudaMemcpyAsync(&gmax, cnt + 12, 4, cudaMemcpyDeviceToHost, st), "gap"));
            FMM_TRY(cuda_check(t, cudaMemcpyAsync(&nd, dense + H, 4, cudaMemcpyDeviceToHost, st), "ndoff"));
            FMM_TRY(cuda_check(t, cudaMemcpyAsync(&inter, inter_d, 8, cudaMemcpyDeviceToHost, st), "p2p count"));
            FMM_TRY(cuda_check(t, cudaMemcpyAsync(&serr, sort_err, 4, cudaMemcpyDeviceToHost, st), "sort status"));
            FMM_TRY(cuda_check(t, cudaStreamSynchronize(st), "sync"));
            if (le) {
                FMM_TRY(layout_radix());
                le = 0;
                continue;
            }
            if (e & kErrKeyRange) {
                t->err = "an accepted M2L offset exceeds 2^16 finer half-cells (theta too small for the tree)";
                return FMM_EINVAL;
            }
            if (!(e & kErrHashFull)) {
                t->max_gap = (int)gmax;
                break;
            }
            H <<= 1;
        }
        uint32_t *dense = (uint32_t *)t->b_scan.ptr;
        ndoff = nd;
        FMM_TRY(ensure(t, t->b_dkeys, 8 * std::max<int64_t>(ndoff, 1)));
        k_slot_compact<<<grid(H, 256), 256, 0, st>>>((unsigned long long *)t->b_hash.ptr, H, dense,
                                                       (uint64_t *)t->b_dkeys.ptr);
        // canonical numbering: keys by value (57-bit keys: gap, side, offsets)
        const int64_t nd1 = std::max<int64_t>(ndoff, 1);
        FMM_TRY(ensure(t, t->b_dsort, 20 * (size_t)nd1));
        FMM_TRY(ensure(t, t->b_dsort_h, radix_hist_bytes(nd1)));
        uint64_t *keys2 = (uint64_t *)t->b_dsort.ptr;
        uint32_t *vals = (uint32_t *)(keys2 + nd1), *vals2 = vals + nd1, *rank_of = vals2 + nd1;
        if (ndoff <= kRankSmall) {
            k_rank_small<<<1, 1024, 8 * (size_t)ndoff, st>>>((uint64_t *)t->b_dkeys.ptr, (int)ndoff, rank_of);
            t->launches += 2;
        } else {
            k_iota<<<grid(ndoff, 256), 256, 0, st>>>(vals, ndoff);
            radix_sort_pairs((uint64_t *)t->b_dkeys.ptr, vals, keys2, vals2, ndoff, 57,
                             (uint32_t *)t->b_dsort_h.ptr, sort_err, st, &t->launches);
            k_rank_of<<<grid(ndoff, 256), 256, 0, st>>>(vals, ndoff, rank_of);
            t->launches += 3;
            dsort = true;
        }
        k_slot_to_dense<<<grid(nm2l, 256), 256, 0, st>>>((int32_t *)t->b_m2l_didx.ptr, nm2l, dense, rank_of);
    }
    // the sort status once more when a radix sort ran after the read above; the
    // long-row flag and the P2P count when there was no M2L list to read them with
    while (nm2l == 0 || dsort) {
        FMM_TRY(cuda_check(t, cudaMemcpyAsync(&serr, sort_err, 4, cudaMemcpyDeviceToHost, st), "sort status"));
        FMM_TRY(cuda_check(t, cudaMemcpyAsync(&le, long_err, 4, cudaMemcpyDeviceToHost, st), "rows"));
        FMM_TRY(cuda_check(t, cudaMemcpyAsync(&inter, inter_d, 8, cudaMemcpyDeviceToHost, st), "p2p count"));
        FMM_TRY(cuda_check(t, cudaStreamSynchronize(st), "sync"));
        if (!le) break;
        FMM_TRY(layout_radix());        // a long P2P row with no M2L list to catch it earlier
    }
    if (serr & kErrSortWait) {
        t->err = "a bounded wait of the radix sort gave up";
        return FMM_ETIMEOUT;
    }
    t->n_m2l = nm2l;
    t->n_p2p = np2p;
    t->n_p2p_inter = (int64_t)inter;
    t->n_doff = ndoff;
    t->theta = theta;
    t->have_lists = true;
    return FMM_OK;
}

}  // namespace fmm
