// m2l32_tile.cu -- the M2L translation of the FMM_FP32 form (and of
// FMM_3XTF32 off the tensor cores) as SIMT FP32 over the tensor-core plan.
//
// The plan of m2l_tc.cu groups the targets 128 to a tile (same level, same
// position in the parent) and, per tile, one row per D key that occurs there:
// the row holds, at each target's lane, the source of that target's pair with
// the key (or none).  All 128 pairs of a row share the operator of Eq. (8) in
// the scaled form, T_key[n][m] = Dh_key[n+m] (h_s/h_t)^(|m|-s), zero where
// |n| + |m| > p + s.  Here one block of 128 threads takes a chunk of rows of a
// tile, thread t the tile's target t: per row it stages the 128 source
// multipole rows (each thread its own, cp.async) and the key's operator image
// in shared memory, then forms L~_t[n] += sum_m T[n][m] M~_s[m] in FP32 with
// the operator read by all lanes at once (one broadcast 16-byte read feeds four
// FMAs of every lane) and the multipole four values to a read.  The locals
// are held in registers in blocks of 8 columns; the columns of block b reach
// the first mb[b] multipoles in graded order (those with |m| <= p + s - the
// block's lowest order), so the triangle costs only the rounding of each
// block.  A chunk's sums (at most G rows, in row order) are written as FP32
// partials, summed over a tile's chunks in double-float by the plan's reduction --
// the accumulation of the tensor-core form, with FP32 products in place of
// 3xTF32.
#include <algorithm>
#include <cstring>

#include "fmm_internal.cuh"
#include "umma.cuh"

namespace fmm {

using namespace umma;

namespace {

constexpr int kT32Threads = 128;     // one thread per target of a tile
constexpr int kT32MaxNB = 16;        // blocks of 8 columns: n_L <= 128
constexpr int kT32SmemMax = 232448;  // dynamic shared memory a block may opt into
constexpr int kT32MaxSeg = 8;        // segments per warp pair of the two-target kernel

struct T32Args {
    const int32_t *chunk_rb, *chunk_re;  // rows [rb, re) of each chunk
    const int32_t *row_key;              // D row of each tile row
    const int32_t *slot;                 // [rows][128] source cell, -1 = none
    const float *M;                      // scaled FP32 multipoles (folded when harmonic), stride ldM
    const float *img;                    // per key: E floats (layout T32Layout)
    float *partial;                      // [chunks][128][Np]
    int nchunks, ldM, nM, nq, E, Np;     // nq = float4 groups of a staged multipole row
    int mb[kT32MaxNB], boff[kT32MaxNB];
    // two-target kernel: the column blocks dealt to the two warp pairs as
    // segments (block, first and end float4 group of multipoles); second = the
    // segment continues a block the other pair began (its sums are added to
    // the other pair's at the chunk's end)
    int nseg[2];
    int seg_b[2][kT32MaxSeg], seg_q0[2][kT32MaxSeg], seg_q1[2][kT32MaxSeg], seg_second[2][kT32MaxSeg];
};

__device__ __forceinline__ void fma8(float (&acc)[8], const float4 &t0, const float4 &t1, float m)
{
    acc[0] = fmaf(t0.x, m, acc[0]);
    acc[1] = fmaf(t0.y, m, acc[1]);
    acc[2] = fmaf(t0.z, m, acc[2]);
    acc[3] = fmaf(t0.w, m, acc[3]);
    acc[4] = fmaf(t1.x, m, acc[4]);
    acc[5] = fmaf(t1.y, m, acc[5]);
    acc[6] = fmaf(t1.z, m, acc[6]);
    acc[7] = fmaf(t1.w, m, acc[7]);
}

// What a stage holds: the row's chunk, whether it is the chunk's last row,
// whether this thread's target has a pair in it; valid = false past the last.
struct T32Row {
    int chunk;
    bool valid, last, has;
};

// NB >= the layout's blocks (those past it have mb = 0 and are not written).
// Shared memory: two stages of [nq][128] float4 multipoles and two of E floats.
// Persistent: block k takes the chunks k, k + grid, ... as one sequence of
// rows, the next row (of this chunk or the next) staged while one is summed;
// a row's source slot and key are loaded a row ahead of its staging, and the
// next chunk's bounds a chunk ahead.
template <int NB>
__global__ void __launch_bounds__(kT32Threads) k_m2l32_tile(const T32Args a)
{
    extern __shared__ float4 sm4[];
    const int tid = threadIdx.x, G = gridDim.x, nch = a.nchunks;
    float4 *Mst = sm4;                                          // [2][nq][128]
    float *Tst = (float *)(sm4 + 2 * a.nq * kT32Threads);       // [2][E]
    float acc[NB][8];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[b][k] = 0.0f;
    // staging cursor: row sr of chunk sj (rows up to sre); the bounds of chunk
    // sj + G and the slot and key of row sr already in registers
    int sj = blockIdx.x;
    if (sj >= nch) return;
    int sr = a.chunk_rb[sj], sre = a.chunk_re[sj];
    int nrb = 0, nre = 0;
    if (sj + G < nch) {
        nrb = a.chunk_rb[sj + G];
        nre = a.chunk_re[sj + G];
    }
    int src = a.slot[(size_t)sr * kT32Threads + tid], key = a.row_key[sr];
    auto stage = [&](int buf) {
        T32Row w;
        w.valid = sj < nch;
        w.chunk = sj;
        w.last = sr + 1 == sre;
        w.has = w.valid && src >= 0;
        if (w.valid) {
            const float *g = a.M + (size_t)max(src, 0) * a.ldM;
            const uint32_t d = smem_u32(Mst + (size_t)buf * a.nq * kT32Threads + tid);
            for (int q = 0; q < a.nq; ++q) {
                const int left = a.nM - 4 * q;
                cp_async16(d + 16u * kT32Threads * q, g + 4 * q, src < 0 ? 0 : 4 * min(left, 4));
            }
            const float *ti = a.img + (size_t)key * a.E;
            const uint32_t td = smem_u32(Tst + (size_t)buf * a.E);
            for (int e = 4 * tid; e < a.E; e += 4 * kT32Threads) cp_async16(td + 4u * e, ti + e, 16);
            // advance the cursor and fetch what the next staging needs
            if (++sr == sre) {
                sj += G;
                sr = nrb;
                sre = nre;
                if (sj + G < nch) {
                    nrb = a.chunk_rb[sj + G];
                    nre = a.chunk_re[sj + G];
                }
            }
            if (sj < nch) {
                src = a.slot[(size_t)sr * kT32Threads + tid];
                key = a.row_key[sr];
            }
        }
        cp_async_commit();                 // an empty group past the last row keeps the count
        return w;
    };
    T32Row cur = stage(0);
    int buf = 0;
    while (cur.valid) {
        const T32Row nxt = stage(buf ^ 1);
        cp_async_wait<1>();
        __syncthreads();
        if (__any_sync(0xffffffffu, cur.has)) {   // a warp whose 32 targets have no pair here skips it
            const float4 *Mb = Mst + (size_t)buf * a.nq * kT32Threads + tid;
            const float4 *Tb = (const float4 *)(Tst + (size_t)buf * a.E);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const float4 *T4 = Tb + (a.boff[b] >> 2);
                const int nqb = a.mb[b] >> 2;
#pragma unroll 2
                for (int q = 0; q < nqb; ++q) {
                    const float4 mv = Mb[q * kT32Threads];
                    fma8(acc[b], T4[8 * q + 0], T4[8 * q + 1], mv.x);
                    fma8(acc[b], T4[8 * q + 2], T4[8 * q + 3], mv.y);
                    fma8(acc[b], T4[8 * q + 4], T4[8 * q + 5], mv.z);
                    fma8(acc[b], T4[8 * q + 6], T4[8 * q + 7], mv.w);
                }
            }
        }
        __syncthreads();                         // before the next row's staging refills the other stage
        if (cur.last) {
            float4 *P = (float4 *)(a.partial + ((size_t)cur.chunk * kT32Threads + tid) * a.Np);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if (8 * b < a.Np) {
                    P[2 * b] = make_float4(acc[b][0], acc[b][1], acc[b][2], acc[b][3]);
                    P[2 * b + 1] = make_float4(acc[b][4], acc[b][5], acc[b][6], acc[b][7]);
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) acc[b][k] = 0.0f;
            }
        }
        cur = nxt;
        buf ^= 1;
    }
    cp_async_wait<0>();
}

// The same sums with two targets per thread: warps 0-1 and 2-3 form two
// pairs; thread u of a pair takes the tile's targets u and u + 64, and each
// pair runs its share of the column blocks (segments of the blocks' multipole
// ranges, about half of the float4 groups each), so every broadcast operator
// value feeds two FMAs.  A block split between the pairs is summed at the
// chunk's end: the first pair writes its part, then the second adds its own.
template <int NS>
__global__ void __launch_bounds__(kT32Threads, 3) k_m2l32_tile2(const T32Args a)
{
    extern __shared__ float4 sm4[];
    __shared__ unsigned char s_has[2][kT32Threads];
    const int tid = threadIdx.x, G = gridDim.x, nch = a.nchunks;
    const int pr = tid >> 6, u = tid & 63;
    float4 *Mst = sm4;                                          // [2][nq][128]
    float *Tst = (float *)(sm4 + 2 * a.nq * kT32Threads);       // [2][E]
    const int nseg = a.nseg[pr];
    float acc[NS][2][8];
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[i][0][k] = acc[i][1][k] = 0.0f;
    int sj = blockIdx.x;
    if (sj >= nch) return;
    int sr = a.chunk_rb[sj], sre = a.chunk_re[sj];
    int nrb = 0, nre = 0;
    if (sj + G < nch) {
        nrb = a.chunk_rb[sj + G];
        nre = a.chunk_re[sj + G];
    }
    int src = a.slot[(size_t)sr * kT32Threads + tid], key = a.row_key[sr];
    // staging as in k_m2l32_tile (each thread its own target's row), plus
    // whether the thread's target has a pair in the row
    auto stage = [&](int buf) {
        T32Row w;
        w.valid = sj < nch;
        w.chunk = sj;
        w.last = sr + 1 == sre;
        w.has = false;
        if (w.valid) {
            s_has[buf][tid] = src >= 0;
            const float *g = a.M + (size_t)max(src, 0) * a.ldM;
            const uint32_t d = smem_u32(Mst + (size_t)buf * a.nq * kT32Threads + tid);
            for (int q = 0; q < a.nq; ++q) {
                const int left = a.nM - 4 * q;
                cp_async16(d + 16u * kT32Threads * q, g + 4 * q, src < 0 ? 0 : 4 * min(left, 4));
            }
            const float *ti = a.img + (size_t)key * a.E;
            const uint32_t td = smem_u32(Tst + (size_t)buf * a.E);
            for (int e = 4 * tid; e < a.E; e += 4 * kT32Threads) cp_async16(td + 4u * e, ti + e, 16);
            if (++sr == sre) {
                sj += G;
                sr = nrb;
                sre = nre;
                if (sj + G < nch) {
                    nrb = a.chunk_rb[sj + G];
                    nre = a.chunk_re[sj + G];
                }
            }
            if (sj < nch) {
                src = a.slot[(size_t)sr * kT32Threads + tid];
                key = a.row_key[sr];
            }
        }
        cp_async_commit();
        return w;
    };
    T32Row cur = stage(0);
    int buf = 0;
    while (cur.valid) {
        const T32Row nxt = stage(buf ^ 1);
        cp_async_wait<1>();
        __syncthreads();
        if (__any_sync(0xffffffffu, s_has[buf][u] | s_has[buf][u + 64])) {
            const float4 *Mb = Mst + (size_t)buf * a.nq * kT32Threads + u;
            const float4 *Tb = (const float4 *)(Tst + (size_t)buf * a.E);
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                if (i < nseg) {
                    const float4 *T4 = Tb + (a.boff[a.seg_b[pr][i]] >> 2);
                    const int q1 = a.seg_q1[pr][i];
#pragma unroll 2
                    for (int q = a.seg_q0[pr][i]; q < q1; ++q) {
                        const float4 m0 = Mb[q * kT32Threads], m1 = Mb[q * kT32Threads + 64];
                        float4 t0 = T4[8 * q + 0], t1 = T4[8 * q + 1];
                        fma8(acc[i][0], t0, t1, m0.x);
                        fma8(acc[i][1], t0, t1, m1.x);
                        t0 = T4[8 * q + 2]; t1 = T4[8 * q + 3];
                        fma8(acc[i][0], t0, t1, m0.y);
                        fma8(acc[i][1], t0, t1, m1.y);
                        t0 = T4[8 * q + 4]; t1 = T4[8 * q + 5];
                        fma8(acc[i][0], t0, t1, m0.z);
                        fma8(acc[i][1], t0, t1, m1.z);
                        t0 = T4[8 * q + 6]; t1 = T4[8 * q + 7];
                        fma8(acc[i][0], t0, t1, m0.w);
                        fma8(acc[i][1], t0, t1, m1.w);
                    }
                }
            }
        }
        __syncthreads();                         // before the next row's staging refills the other stage
        if (cur.last) {
            float *P = a.partial + (size_t)cur.chunk * kT32Threads * a.Np;
            // first parts (and whole blocks), then the second parts added to them
            for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
                for (int i = 0; i < NS; ++i) {
                    if (i < nseg && a.seg_second[pr][i] == pass) {
                        const int c0 = 8 * a.seg_b[pr][i];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            float4 *d = (float4 *)(P + (size_t)(u + 64 * h) * a.Np + c0);
                            float4 v0 = make_float4(acc[i][h][0], acc[i][h][1], acc[i][h][2], acc[i][h][3]);
                            float4 v1 = make_float4(acc[i][h][4], acc[i][h][5], acc[i][h][6], acc[i][h][7]);
                            if (pass == 1) {
                                const float4 w0 = d[0], w1 = d[1];
                                v0 = make_float4(w0.x + v0.x, w0.y + v0.y, w0.z + v0.z, w0.w + v0.w);
                                v1 = make_float4(w1.x + v1.x, w1.y + v1.y, w1.z + v1.z, w1.w + v1.w);
                            }
                            d[0] = v0;
                            d[1] = v1;
                        }
                    }
                }
                __syncthreads();                 // the first parts are visible to the block
            }
#pragma unroll
            for (int i = 0; i < NS; ++i)
#pragma unroll
                for (int k = 0; k < 8; ++k) acc[i][0][k] = acc[i][1][k] = 0.0f;
        }
        cur = nxt;
        buf ^= 1;
    }
    cp_async_wait<0>();
}

// operator images: float e of key r's image is the D entry el_src[e] with the
// key's power-of-two scalings (the target's side for the order of n + m, the
// level gap for |m| - s), rounded once to FP32; zero where el_src[e] < 0
__global__ void k_m32_images(int64_t ndoff, int E, const uint64_t *dkeys, const double *D, int nD,
                             const int32_t *el_src, float *img)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= ndoff * E) return;
    const int64_t r = g / E;
    const int src = el_src[g - r * E];
    float v = 0.0f;
    if (src >= 0) {
        const uint64_t key = dkeys[r];
        const int gap = (int)((key >> 52) & 31), tfiner = (int)((key >> 51) & 1);
        const int esc = tfiner ? 0 : gap, dl = tfiner ? gap : -gap;
        const int k = src & 0xFFFF, nm = (src >> 16) & 0xFF, msh = src >> 24;
        v = (float)ldexp(D[r * nD + k], (nm + 1) * esc + dl * msh);
    }
    img[g] = v;
}

void build_layout32(T32Layout &Ly, int s, int p, int h, int n_lo)
{
    const MultiIndex &I = multi_index();
    auto shell = [&](int k) { return I.nx[k] + I.ny[k] + I.nz[k]; };
    std::vector<int> ms, ns;
    for (int k = ntot(s - 1); k < ntot(p + s); ++k)
        if (!h || I.nz[k] <= 1) ms.push_back(k);
    for (int n = 0; n < ntot(p); ++n)
        if (shell(n) >= n_lo && (!h || I.nz[n] <= 1)) ns.push_back(n);
    Ly.s = s;
    Ly.p = p;
    Ly.h = h;
    Ly.n_lo = n_lo;
    Ly.nM = (int)ms.size();
    Ly.ncol = (int)ns.size();
    Ly.col_n = ns;
    Ly.nb = (Ly.ncol + 7) / 8;
    Ly.Np = 8 * Ly.nb;
    const int nMp = (Ly.nM + 3) & ~3;
    Ly.mb.assign(Ly.nb, 0);
    Ly.boff.assign(Ly.nb, 0);
    int off = 0;
    for (int b = 0; b < Ly.nb; ++b) {
        const int reach = p + s - shell(ns[8 * b]);     // graded: the block's lowest order comes first
        int cnt = 0;
        while (cnt < Ly.nM && shell(ms[cnt]) <= reach) ++cnt;
        Ly.mb[b] = std::min((cnt + 3) & ~3, nMp);
        Ly.boff[b] = off;
        off += 8 * Ly.mb[b];
    }
    Ly.E = off;
    Ly.el_src.assign(Ly.E, -1);
    for (int b = 0; b < Ly.nb; ++b)
        for (int m = 0; m < Ly.mb[b]; ++m)
            for (int jj = 0; jj < 8; ++jj) {
                const int col = 8 * b + jj;
                if (col >= Ly.ncol || m >= Ly.nM) continue;
                const int n = ns[col], gm = ms[m], tot = shell(n) + shell(gm);
                if (tot > p + s) continue;
                const int d = I(I.nx[n] + I.nx[gm], I.ny[n] + I.ny[gm], I.nz[n] + I.nz[gm]);
                Ly.el_src[Ly.boff[b] + 8 * m + jj] = d | tot << 16 | (shell(gm) - s) << 24;
            }
}

inline size_t t32_smem(const T32Layout &Ly)
{
    const size_t nq = (size_t)(Ly.nM + 3) / 4;
    return 2 * 16 * nq * kT32Threads + 2 * 4 * (size_t)Ly.E;
}

inline unsigned gridn(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

bool m32_usable(fmm_tree *t, int s, int p, int harmonic, int n_lo)
{
    T32Layout &Ly = t->m32_lay;
    const int h = harmonic ? 1 : 0;
    if (Ly.s != s || Ly.p != p || Ly.h != h || Ly.n_lo != n_lo) {
        build_layout32(Ly, s, p, h, n_lo);
        t->m32_img_p = -1;                    // images and element map of the old layout
    }
    return Ly.ncol > 0 && Ly.nb <= kT32MaxNB && t32_smem(Ly) <= (size_t)kT32SmemMax;
}

fmm_status m32_prepare(fmm_tree *t, int p)
{
    cudaStream_t st = t->stream;
    const T32Layout &Ly = t->m32_lay;
    if (!t->tc_plan) FMM_TRY(tc_build_plan(t));
    if (t->tc_chunks == 0) return FMM_OK;
    if (t->m32_img_p != p) {
        FMM_TRY(ensure(t, t->b_m32_el, 4 * ((size_t)Ly.E + Ly.ncol)));
        FMM_TRY(cuda_check(t, cudaMemcpyAsync(t->b_m32_el.ptr, Ly.el_src.data(), 4 * (size_t)Ly.E,
                                              cudaMemcpyHostToDevice, st), "upload"));
        FMM_TRY(cuda_check(t, cudaMemcpyAsync((int32_t *)t->b_m32_el.ptr + Ly.E, Ly.col_n.data(),
                                              4 * (size_t)Ly.ncol, cudaMemcpyHostToDevice, st), "upload"));
        FMM_TRY(ensure(t, t->b_m32_img, 4 * (size_t)t->n_doff * Ly.E));
        k_m32_images<<<gridn(t->n_doff * Ly.E, 256), 256, 0, st>>>(
            t->n_doff, Ly.E, (const uint64_t *)t->b_dkeys.ptr, (const double *)t->b_D.ptr, ntot(p + t->s),
            (const int32_t *)t->b_m32_el.ptr, (float *)t->b_m32_img.ptr);
        ++t->launches;
        t->m32_img_p = p;
    }
    return ensure(t, t->b_tc_part, 4 * (size_t)t->tc_chunks * kT32Threads * Ly.Np);
}

fmm_status run_m2l32_tile(fmm_tree *t, int p, const float *M, int ldM, const DevTables &tb, float *L)
{
    cudaStream_t st = t->stream;
    const T32Layout &Ly = t->m32_lay;
    if ((Ly.h == 1) != (tb.harmonic == 1) || Ly.nM != tb.nMh || ldM % 4 != 0) {
        t->err = "tiled FP32 M2L: layout and tables disagree";
        return FMM_EINVAL;                   // not reachable: both follow the handle's flag
    }
    if (!t->tc_plan || t->m32_img_p != p) FMM_TRY(m32_prepare(t, p));
    if (t->tc_chunks == 0) return FMM_OK;
    T32Args a;
    std::memset(&a, 0, sizeof(a));
    a.chunk_rb = (const int32_t *)t->b_tc_crb.ptr;
    a.chunk_re = (const int32_t *)t->b_tc_cre.ptr;
    a.row_key = (const int32_t *)t->b_tc_rowkey.ptr;
    a.slot = (const int32_t *)t->b_tc_slot.ptr;
    a.M = M;
    a.img = (const float *)t->b_m32_img.ptr;
    a.partial = (float *)t->b_tc_part.ptr;
    a.ldM = ldM;
    a.nM = Ly.nM;
    a.nq = (Ly.nM + 3) / 4;
    a.E = Ly.E;
    a.Np = Ly.Np;
    a.nchunks = (int)t->tc_chunks;
    for (int b = 0; b < Ly.nb; ++b) {
        a.mb[b] = Ly.mb[b];
        a.boff[b] = Ly.boff[b];
    }
    // two targets per thread where the blocks' float4 groups split evenly into
    // at most kT32MaxSeg segments per warp pair (in block order: the first
    // pair takes the blocks up to half the groups, the block at the boundary
    // split between the pairs)
    int Q = 0;
    for (int b = 0; b < Ly.nb; ++b) Q += Ly.mb[b] / 4;
    const int halfQ = (Q + 1) / 2;
    bool two = true;
    auto add = [&](int pr, int b, int q0, int q1, int second) {
        int &n = a.nseg[pr];
        if (n >= kT32MaxSeg) {
            two = false;
            return;
        }
        a.seg_b[pr][n] = b;
        a.seg_q0[pr][n] = q0;
        a.seg_q1[pr][n] = q1;
        a.seg_second[pr][n] = second;
        ++n;
    };
    for (int b = 0, pr = 0, acc = 0; b < Ly.nb; ++b) {
        const int qn = Ly.mb[b] / 4;
        if (pr == 0 && acc + qn > halfQ) {
            const int take = halfQ - acc;
            if (take > 0) {
                add(0, b, 0, take, 0);
                add(1, b, take, qn, 1);
            } else {
                add(1, b, 0, qn, 0);
            }
            pr = 1;
            continue;
        }
        add(pr, b, 0, qn, 0);
        acc += qn;
    }
    const size_t smem = t32_smem(Ly);
    auto go = [&](auto kern) {
        allow_max_dynamic_smem(kern);
        // persistent: as many blocks as are resident at once, at most one per chunk
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT32Threads, smem) != cudaSuccess)
            per_sm = 1;
        const int64_t grid = std::min<int64_t>(t->tc_chunks, (int64_t)std::max(per_sm, 1) * sm_count());
        kern<<<(unsigned)grid, kT32Threads, smem, st>>>(a);
    };
    const int ns = std::max(a.nseg[0], a.nseg[1]);
    if (two && ns <= 2) go(k_m2l32_tile2<2>);
    else if (two && ns <= 4) go(k_m2l32_tile2<4>);
    else if (two && ns <= 6) go(k_m2l32_tile2<6>);
    else if (two) go(k_m2l32_tile2<8>);
    else switch ((Ly.nb + 1) / 2) {
    case 1: go(k_m2l32_tile<2>); break;
    case 2: go(k_m2l32_tile<4>); break;
    case 3: go(k_m2l32_tile<6>); break;
    case 4: go(k_m2l32_tile<8>); break;
    case 5: go(k_m2l32_tile<10>); break;
    case 6: go(k_m2l32_tile<12>); break;
    case 7: go(k_m2l32_tile<14>); break;
    default: go(k_m2l32_tile<16>); break;
    }
    ++t->launches;
    // the reduction reads the tensor-core timeout flag: none here
    unsigned *err = (unsigned *)t->b_err.ptr + 1;
    cudaMemsetAsync(err, 0, sizeof(unsigned), st);
    launch_tc_reduce(t, Ly.Np, Ly.ncol, (const int32_t *)t->b_m32_el.ptr + Ly.E, tb.nL, tb, err, L);
    return cuda_check(t, cudaGetLastError(), "tiled FP32 M2L");
}

}  // namespace fmm
