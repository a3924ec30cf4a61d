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
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            atomicMin(&box[d], mn[d]);
            atomicMax(&box[3 + d], mx[d]);
        }
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

__global__ void k_keys(const double *pos, int64_t n, const double *box, uint64_t *keys,
                       uint32_t *idx)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double scale = ldexp(1.0, kLevels) / box[3];      // a power of two
    uint64_t q[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double u = floor(__dmul_rn(__dsub_rn(pos[3 * i + d], box[d]), scale));
        uint64_t v = (uint64_t)u;
        q[d] = v > (uint64_t)((1 << kLevels) - 1) ? (uint64_t)((1 << kLevels) - 1) : v;
    }
    keys[i] = spread3(q[0]) << 2 | spread3(q[1]) << 1 | spread3(q[2]);
    idx[i] = (uint32_t)i;
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

// child ranges of every (cell of this level, octant), and each cell's child count
__global__ void __launch_bounds__(256)
k_level_ranges(CellArrays c, const unsigned *ctl, int level, int ncrit, const uint64_t *keys,
               int32_t *cb, int32_t *ce, uint32_t *cnt)
{
    if (ctl[kCtlOverflow]) return;
    const int lb = (int)ctl[kCtlLevel + level];
    const int64_t n8 = 8 * ((int64_t)ctl[kCtlLevel + level + 1] - lb);
    const unsigned lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n8; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = base + threadIdx.x;
        bool flag = false;
        if (t < n8) {
            const int cell = lb + (int)(t >> 3), o = (int)(t & 7);
            const int b = c.begin[cell], e = c.end[cell];
            int lo_i = b, hi_i = b;
            if (e - b > ncrit && level < kLevels) {
                // first index in [b, e) whose child digit is >= o (resp. >= o + 1)
                int L = b, R = e;
                while (L < R) {
                    const int mid = (L + R) >> 1;
                    if (digit_at(keys[mid], level + 1) < o) L = mid + 1; else R = mid;
                }
                lo_i = L;
                R = e;
                while (L < R) {
                    const int mid = (L + R) >> 1;
                    if (digit_at(keys[mid], level + 1) <= o) L = mid + 1; else R = mid;
                }
                hi_i = L;
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
    for (int base = 0; base < ncl; base += 8 * (int)blockDim.x) {
        const int i0 = base + 8 * (int)threadIdx.x;
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            v[k] = i0 + k < ncl ? cnt[i0 + k] : 0u;
            sum += v[k];
        }
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
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (i0 + k < ncl) off[i0 + k] = ex;
            ex += v[k];
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

__global__ void k_cell_geometry(CellArrays c, int64_t ncells, const double *box, double *centre,
                                double *half, uint32_t *leaf_flag)
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
}

__global__ void k_compact_leaves(const uint32_t *flag, const uint32_t *pos, int64_t ncells,
                                 int32_t *leaves)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < ncells && flag[i]) leaves[pos[i]] = (int32_t)i;
}

// ----------------------------------------------------------- traversal
// MAC of Eq. (13), exact: centres (2c+1) 2^(21-l) and radii 2^(21-l) in units
// of the finest half-cell; (rA + rB)^2 < (theta*theta) |dc|^2.
__device__ __forceinline__ bool mac_accept(const CellArrays &c, int a, int b, double theta2)
{
    const int la = c.level[a], lb = c.level[b];
    const long long ra = 1ll << (kLevels - la), rb = 1ll << (kLevels - lb);
    const long long dx = (2ll * c.cx[a] + 1) * ra - (2ll * c.cx[b] + 1) * rb;
    const long long dy = (2ll * c.cy[a] + 1) * ra - (2ll * c.cy[b] + 1) * rb;
    const long long dz = (2ll * c.cz[a] + 1) * ra - (2ll * c.cz[b] + 1) * rb;
    const long long d2 = dx * dx + dy * dy + dz * dz;
    const double lhs = (double)((ra + rb) * (ra + rb));
    return lhs < __dmul_rn(theta2, (double)d2);
}

// Warp-aggregated reservation: every lane asks for `want` slots of one list;
// one atomic per warp, lanes get consecutive ranges in lane order.
__device__ __forceinline__ unsigned warp_reserve(unsigned *count, unsigned want)
{
    const int lane = threadIdx.x & 31;
    unsigned incl = want;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned base = 0;
    if (lane == 31 && total) base = atomicAdd(count, total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + incl - want;
}

// One round of the breadth-first dual traversal.  The rounds are launched
// back to back without the host: round r reads its frontier size from
// counters[kTravFront + r] and adds the next round's to the word after it.
// counters: 0 = m2l, 1 = p2p, kTravOverflow = a frontier exceeded front_cap
// (every later round then does nothing).  Outputs beyond a list's capacity
// are counted but not written; the host grows what overflowed and reruns
// the whole traversal.
constexpr int kTravOverflow = 16, kTravFront = 32, kTravMaxRounds = 960;
// blocks of a traversal round: 8 resident blocks of 256 threads per SM
constexpr int kTravBlocksPerSM = 8;

__global__ void __launch_bounds__(256)
k_traverse_round(CellArrays c, int round, double theta2, const int2 *front, unsigned front_cap,
                 int2 *m2l, unsigned m2l_cap, int2 *p2p, unsigned p2p_cap, int2 *next,
                 unsigned *counters)
{
    const unsigned nf = counters[kTravFront + round];
    if (nf == 0 || counters[kTravOverflow]) return;
    if (nf > front_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&counters[kTravOverflow], 1u);
        return;
    }
    unsigned *next_count = &counters[kTravFront + round + 1];
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned base = blockIdx.x * blockDim.x; base < nf; base += stride) {
        const unsigned t = base + threadIdx.x;
        const bool valid = t < nf;
        int a = 0, b = 0, na = 0, nb = 0;
        if (valid) {
            a = front[t].x; b = front[t].y;
            na = c.nchild[a]; nb = c.nchild[b];
        }
        // classify: kind 0 = M2L, 1 = P2P, 2 = open a (all children against b,
        // or all child pairs for a self pair), 3 = open b
        int kind = -1;
        if (valid) {
            if (a == b) kind = na == 0 ? 1 : 2;
            else if (mac_accept(c, a, b, theta2)) kind = 0;
            else if (na == 0 && nb == 0) kind = 1;
            else if (na == 0) kind = 3;
            else if (nb == 0) kind = 2;
            else kind = c.level[a] <= c.level[b] ? 2 : 3;
        }
        const unsigned n_next = kind == 2 ? (a == b ? (unsigned)(na * na) : (unsigned)na)
                                          : (kind == 3 ? (unsigned)nb : 0u);
        const unsigned o_m2l = warp_reserve(&counters[0], kind == 0);
        const unsigned o_p2p = warp_reserve(&counters[1], kind == 1);
        const unsigned o_next = warp_reserve(next_count, n_next);
        if (kind == 0) {
            if (o_m2l < m2l_cap) m2l[o_m2l] = make_int2(a, b);
        } else if (kind == 1) {
            if (o_p2p < p2p_cap) p2p[o_p2p] = make_int2(a, b);
        } else if (kind == 2) {
            const int f = c.child[a];
            if (a == b) {
                for (int i = 0; i < na; ++i)
                    for (int j = 0; j < na; ++j) {
                        const unsigned k = o_next + (unsigned)(i * na + j);
                        if (k < front_cap) next[k] = make_int2(f + i, f + j);
                    }
            } else {
                for (int i = 0; i < na; ++i)
                    if (o_next + i < front_cap) next[o_next + i] = make_int2(f + i, b);
            }
        } else if (kind == 3) {
            const int f = c.child[b];
            for (int j = 0; j < nb; ++j)
                if (o_next + j < front_cap) next[o_next + j] = make_int2(a, f + j);
        }
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

__global__ void k_offset_keys(CellArrays c, const uint64_t *pair_keys, int64_t np, int cbits,
                              unsigned long long *table, uint32_t hmask, uint32_t *slot_of,
                              int *err, unsigned *max_gap)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= np) return;
    const int a = (int)(pair_keys[k] >> cbits), b = (int)(pair_keys[k] & ((1ull << cbits) - 1ull));
    const int la = c.level[a], lb = c.level[b], lf = la > lb ? la : lb;
    const long long sa = 1ll << (lf - la), sb = 1ll << (lf - lb);
    long long d[3] = {(2ll * c.cx[a] + 1) * sa - (2ll * c.cx[b] + 1) * sb,
                      (2ll * c.cy[a] + 1) * sa - (2ll * c.cy[b] + 1) * sb,
                      (2ll * c.cz[a] + 1) * sa - (2ll * c.cz[b] + 1) * sb};
    const int gap = la > lb ? la - lb : lb - la;
    if (gap) atomicMax(max_gap, (unsigned)gap);
    uint64_t key = (uint64_t)gap << 52 | (uint64_t)(la > lb) << 51;
    for (int i = 0; i < 3; ++i) {
        if (d[i] < -kKeyBias || d[i] >= kKeyBias) { atomicOr(err, kErrKeyRange); slot_of[k] = 0; return; }
        key |= (uint64_t)(d[i] + kKeyBias) << (34 - 17 * i);
    }
    uint32_t h = (uint32_t)hash64(key) & hmask;
    for (uint32_t probe = 0; probe <= hmask; ++probe) {
        unsigned long long cur = table[h];
        if (cur == key) { slot_of[k] = h; return; }
        if (cur == ~0ull) {
            unsigned long long prev = atomicCAS(&table[h], ~0ull, (unsigned long long)key);
            if (prev == ~0ull || prev == key) { slot_of[k] = h; return; }
        }
        h = (h + 1) & hmask;
    }
    atomicOr(err, kErrHashFull);
    slot_of[k] = 0;
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
static void morton_keys(cudaStream_t st, const double *pos, int64_t n, uint64_t *keys,
                        uint32_t *idx, unsigned long long *box_scratch, double *box_out, int *err,
                        int64_t *launches)
{
    k_box_init<<<1, 32, 0, st>>>(box_scratch);
    k_bbox<<<(unsigned)std::min<int64_t>(grid(n, 256), 8 * (int64_t)sm_count()), 256, 0, st>>>(pos, n, box_scratch, err);
    k_box_final<<<1, 1, 0, st>>>(box_scratch, box_out);
    k_keys<<<grid(n, 256), 256, 0, st>>>(pos, n, box_out, keys, idx);
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
    morton_keys(st, pos, n, keys, idx, box_scratch, box_out, err, launches);
    radix_sort_pairs(keys, idx, keys2, idx2, n, 3 * kLevels, hist, err, st, launches);
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
        morton_keys(st, pos, n, keys, idx, sbox_raw, sbox, (int *)t->b_err.ptr, &t->launches);
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
                     3 * kLevels, (uint32_t *)t->b_hist.ptr, (int *)t->b_err.ptr, st, &t->launches);
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
    k_cell_geometry<<<grid(nc, 256), 256, 0, st>>>(c, nc, sbox, (double *)t->b_centre.ptr,
                                                    (double *)t->b_half.ptr, flags);
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
    const int nsys = (int)t->sys_off.size() - 1;
    size_t m2l_cap = std::max<size_t>(4096, t->m2l_cap_hint), p2p_cap = std::max<size_t>(4096, 40 * (size_t)t->nleaves);
    size_t front_cap = std::max<size_t>({(size_t)4096, (size_t)nsys, 16 * (size_t)t->nleaves,
                                         t->b_front.bytes / 8, t->b_front2.bytes / 8});
    std::vector<unsigned> hc((size_t)kTravFront + kTravMaxRounds + 1);
    const int batch = 2 * std::max(t->nlevels, 1) + 1;
    for (;;) {
        FMM_TRY(grow_keep(t, t->b_m2l_raw, 8 * m2l_cap, 0));
        FMM_TRY(grow_keep(t, t->b_p2p_raw, 8 * p2p_cap, 0));
        FMM_TRY(grow_keep(t, t->b_front, 8 * front_cap, 0));
        FMM_TRY(grow_keep(t, t->b_front2, 8 * front_cap, 0));
        m2l_cap = t->b_m2l_raw.bytes / 8;
        p2p_cap = t->b_p2p_raw.bytes / 8;
        front_cap = std::min(t->b_front.bytes, t->b_front2.bytes) / 8;
        int2 *fr[2] = {(int2 *)t->b_front.ptr, (int2 *)t->b_front2.ptr};
        FMM_TRY(cuda_check(t, cudaMemsetAsync(cnt, 0, 4 * (kTravFront + kTravMaxRounds + 1), st),
                           "counters"));
        k_root_pairs<<<grid(nsys, 128), 128, 0, st>>>(fr[0], nsys, cnt + kTravFront);
        ++t->launches;
        int r = 0;
        bool retry = false;
        const unsigned trav_blocks = (unsigned)(kTravBlocksPerSM * sm_count());
        for (;;) {
            const int end = std::min(r + batch, kTravMaxRounds);
            for (; r < end; ++r) {
                k_traverse_round<<<trav_blocks, 256, 0, st>>>(
                    c, r, theta2, fr[r & 1], (unsigned)front_cap, (int2 *)t->b_m2l_raw.ptr,
                    (unsigned)m2l_cap, (int2 *)t->b_p2p_raw.ptr, (unsigned)p2p_cap, fr[(r + 1) & 1], cnt);
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

    // ---- sort both lists by (target, source) and build CSR offsets
    int cbits = 1;
    while ((1ll << cbits) < nc) ++cbits;
    const int64_t nmax = std::max(nm2l, np2p);
    FMM_TRY(ensure(t, t->b_lkeys, 8 * std::max<int64_t>(nmax, 1)));
    FMM_TRY(ensure(t, t->b_lkeys2, 8 * std::max<int64_t>(nmax, 1)));
    FMM_TRY(ensure(t, t->b_lval, 4 * std::max<int64_t>(nmax, 1)));
    FMM_TRY(ensure(t, t->b_lval2, 4 * std::max<int64_t>(nmax, 1)));
    FMM_TRY(ensure(t, t->b_hist, radix_hist_bytes(nmax)));
    FMM_TRY(ensure(t, t->b_scan_tmp, scan_scratch_bytes(std::max<int64_t>(nmax, 1 << 20) * 8)));
    FMM_TRY(ensure(t, t->b_m2l_src, 4 * std::max<int64_t>(nm2l, 1)));
    FMM_TRY(ensure(t, t->b_m2l_didx, 4 * std::max<int64_t>(nm2l, 1)));
    FMM_TRY(ensure(t, t->b_m2l_off, 4 * (nc + 1)));
    FMM_TRY(ensure(t, t->b_p2p_src, 4 * std::max<int64_t>(np2p, 1)));
    FMM_TRY(ensure(t, t->b_p2p_off, 4 * (nc + 1)));
    uint64_t *lk = (uint64_t *)t->b_lkeys.ptr, *lk2 = (uint64_t *)t->b_lkeys2.ptr;
    uint32_t *lv = (uint32_t *)t->b_lval.ptr, *lv2 = (uint32_t *)t->b_lval2.ptr;

    // P2P first (its keys are not needed afterwards except for the count);
    // the sorts report a wait that gave up in counter word 14
    int *sort_err = (int *)(cnt + 14);
    cudaMemsetAsync(sort_err, 0, 4, st);
    k_pack_pairs<<<grid(np2p, 256), 256, 0, st>>>((const int2 *)t->b_p2p_raw.ptr, np2p, cbits, lk, lv);
    radix_sort_pairs(lk, lv, lk2, lv2, np2p, 2 * cbits, (uint32_t *)t->b_hist.ptr, sort_err, st,
                     &t->launches);
    k_row_offsets<<<grid(nc + 1, 256), 256, 0, st>>>(lk, np2p, cbits, nc, (int32_t *)t->b_p2p_off.ptr);
    k_unpack_src<<<grid(np2p, 256), 256, 0, st>>>(lk, np2p, cbits, (int32_t *)t->b_p2p_src.ptr);
    cudaMemsetAsync(cnt + 8, 0, 8, st);
    k_p2p_interactions<<<grid(np2p, 256), 256, 0, st>>>(lk, np2p, cbits, c,
                                                        (unsigned long long *)(cnt + 8));
    t->launches += 4;
    unsigned long long inter = 0;
    FMM_TRY(cuda_check(t, cudaMemcpyAsync(&inter, cnt + 8, 8, cudaMemcpyDeviceToHost, st), "p2p count"));

    // M2L
    if (nm2l > 0) {
        k_pack_pairs<<<grid(nm2l, 256), 256, 0, st>>>((const int2 *)t->b_m2l_raw.ptr, nm2l, cbits, lk, lv);
        radix_sort_pairs(lk, lv, lk2, lv2, nm2l, 2 * cbits, (uint32_t *)t->b_hist.ptr, sort_err,
                         st, &t->launches);
        k_unpack_src<<<grid(nm2l, 256), 256, 0, st>>>(lk, nm2l, cbits, (int32_t *)t->b_m2l_src.ptr);
        t->launches += 2;
    }
    k_row_offsets<<<grid(nc + 1, 256), 256, 0, st>>>(lk, nm2l, cbits, nc, (int32_t *)t->b_m2l_off.ptr);
    ++t->launches;

    // ---- distinct M2L offsets (rows of the derivative table)
    int64_t ndoff = 0;
    if (nm2l > 0) {
        uint32_t H = 1u << 16;
        while (H < 4 * (uint32_t)std::min<int64_t>(nm2l, 1 << 22) && H < (1u << 20)) H <<= 1;
        cudaMemsetAsync(cnt + 12, 0, 4, st);
        for (;;) {
            FMM_TRY(ensure(t, t->b_hash, 8 * (size_t)H));
            FMM_TRY(ensure(t, t->b_flags, 4 * ((size_t)H + 1)));
            FMM_TRY(ensure(t, t->b_scan, 4 * ((size_t)H + 1)));
            cudaMemsetAsync(t->b_hash.ptr, 0xff, 8 * (size_t)H, st);
            cudaMemsetAsync(t->b_err.ptr, 0, sizeof(int), st);
            k_offset_keys<<<grid(nm2l, 256), 256, 0, st>>>(c, lk, nm2l, cbits,
                                                            (unsigned long long *)t->b_hash.ptr,
                                                            H - 1, (uint32_t *)t->b_m2l_didx.ptr,
                                                            (int *)t->b_err.ptr, cnt + 12);
            ++t->launches;
            int e = 0;
            FMM_TRY(cuda_check(t, cudaMemcpyAsync(&e, t->b_err.ptr, 4, cudaMemcpyDeviceToHost, st), "err"));
            FMM_TRY(cuda_check(t, cudaStreamSynchronize(st), "sync"));
            if (e & kErrKeyRange) {
                t->err = "an accepted M2L offset exceeds 2^16 finer half-cells (theta too small for the tree)";
                return FMM_EINVAL;
            }
            if (!(e & kErrHashFull)) break;
            H <<= 1;
        }
        uint32_t *flag = (uint32_t *)t->b_flags.ptr, *dense = (uint32_t *)t->b_scan.ptr;
        cudaMemsetAsync(flag + H, 0, 4, st);
        k_slot_flags<<<grid(H, 256), 256, 0, st>>>((unsigned long long *)t->b_hash.ptr, H, flag);
        exclusive_scan_u32(flag, dense, (int64_t)H + 1, (uint32_t *)t->b_scan_tmp.ptr, st, &t->launches);
        uint32_t nd = 0;
        unsigned gmax = 0;
        FMM_TRY(cuda_check(t, cudaMemcpyAsync(&gmax, cnt + 12, 4, cudaMemcpyDeviceToHost, st), "gap"));
        FMM_TRY(cuda_check(t, cudaMemcpyAsync(&nd, dense + H, 4, cudaMemcpyDeviceToHost, st), "ndoff"));
        FMM_TRY(cuda_check(t, cudaStreamSynchronize(st), "sync"));
        ndoff = nd;
        t->max_gap = (int)gmax;
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
        }
        k_slot_to_dense<<<grid(nm2l, 256), 256, 0, st>>>((int32_t *)t->b_m2l_didx.ptr, nm2l, dense, rank_of);
    }
    int serr = 0;
    FMM_TRY(cuda_check(t, cudaMemcpyAsync(&serr, sort_err, 4, cudaMemcpyDeviceToHost, st), "sort status"));
    FMM_TRY(cuda_check(t, cudaStreamSynchronize(st), "sync"));
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
