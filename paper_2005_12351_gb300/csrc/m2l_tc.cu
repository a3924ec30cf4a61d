// m2l_tc.cu -- the M2L translation of the FMM_3XTF32 form on the tcgen05
// tensor cores, and a self-check of the tensor-core building blocks.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "df32.cuh"
#include "fmm_internal.cuh"
#include "umma.cuh"

namespace fmm {

using namespace umma;

namespace {

// ------------------------------------------------------------ self-check
// One block: D[128 x N] = sum over K-blocks kb of A[:, kb] . B[:N_kb, kb]^T,
// with A [128 x 8 nkb] and B [N x 8 nkb] FP32 row-major, each split into
// two TF32 halves; passes = 1 forms hi.hi only, passes = 3 adds hi.lo and
// lo.hi.  A is staged in shared memory or (a_tmem) in tensor memory.
struct CheckArgs {
    int nkb, N, a_tmem, passes;
    int kbn[4];
};

constexpr int kCheckBBytes = 4 * 2 * 256 * 32;   // 4 K-blocks of hi + lo, N <= 256

__global__ void __launch_bounds__(128) k_check_umma(const float *A, const float *B, float *D, CheckArgs a,
                                                     unsigned *err)
{
    extern __shared__ uint8_t sm_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, K = 8 * a.nkb, N = a.N;
    uint8_t *Asm = sm;                            // per K-block: hi 4 KB, lo 4 KB
    uint8_t *Bsm = sm + 32768;                    // per K-block: hi N x 32 B, lo N x 32 B
    uint64_t *bar = (uint64_t *)(sm + 32768 + kCheckBBytes);
    uint32_t *tslot = (uint32_t *)(bar + 1);
    volatile int *abort = (volatile int *)(tslot + 1);
    if (tid == 0) {
        mbar_init(smem_u32(bar), 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tslot), 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
    // A: thread tid owns row tid
    for (int kb = 0; kb < a.nkb; ++kb) {
        float hi[8], lo[8];
        for (int k = 0; k < 8; ++k) split_tf32(A[tid * K + 8 * kb + k], hi[k], lo[k]);
        if (a.a_tmem) {
            tmem_st8(tmem + lane_off + 256 + 8 * kb, hi);
            tmem_st8(tmem + lane_off + 384 + 8 * kb, lo);
        } else {
            for (int c = 0; c < 2; ++c) {
                *(float4 *)(Asm + kb * 8192 + swz32(tid, c)) =
                    make_float4(hi[4 * c], hi[4 * c + 1], hi[4 * c + 2], hi[4 * c + 3]);
                *(float4 *)(Asm + kb * 8192 + 4096 + swz32(tid, c)) =
                    make_float4(lo[4 * c], lo[4 * c + 1], lo[4 * c + 2], lo[4 * c + 3]);
            }
        }
    }
    // B: element (n, k) of K-block kb
    for (int e = tid; e < N * K; e += 128) {
        const int n = e / K, k = e % K, kb = k >> 3, kk = k & 7;
        float hi, lo;
        split_tf32(B[e], hi, lo);
        const uint32_t off = kb * 64 * N + swz32(n, kk >> 2) + (kk & 3) * 4;
        *(float *)(Bsm + off) = hi;
        *(float *)(Bsm + off + 32 * N) = lo;
    }
    fence_async_smem();
    if (a.a_tmem) tmem_wait_st();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
        for (int kb = 0; kb < a.nkb; ++kb) {
            const uint32_t idesc = idesc_tf32_m128(a.kbn[kb]);
            const uint32_t bh = smem_u32(Bsm + kb * 64 * N);
            for (int pass = 0; pass < a.passes; ++pass) {
                const bool ahi = pass != 2, bhi = pass != 1;
                const uint64_t bd = sdesc_sw32(bhi ? bh : bh + 32 * N);
                const uint32_t acc = (kb > 0 || pass > 0) ? 1u : 0u;
                if (a.a_tmem)
                    mma_tf32_ts(tmem, tmem + (ahi ? 256 : 384) + 8 * kb, bd, idesc, acc);
                else
                    mma_tf32_ss(tmem, sdesc_sw32(smem_u32(Asm + kb * 8192 + (ahi ? 0 : 4096))), bd, idesc,
                                acc);
            }
        }
        mma_commit(smem_u32(bar));
    }
    mbar_wait(smem_u32(bar), 0, abort);
    __syncthreads();
    const bool ok = *abort == 0;
    if (ok) {
        tc_fence_after();
        for (int c0 = 0; c0 < N; c0 += 8) {
            float v[8];
            tmem_ld8(tmem + lane_off + c0, v);
            for (int j = 0; j < 8; ++j) D[tid * N + c0 + j] = v[j];
        }
    } else if (tid == 0) {
        atomicOr(err, 1u);
        // the MMAs may still be running: free tensor memory only after their commit
        mbar_wait_cleanup(smem_u32(bar), 0);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}


// ------------------------------------------------------------------ M2L
// For a fixed D key (level gap, which side is finer, integer offset) the
// translation of Eq. (8) in the scaled form of the mixed-precision path is
// a matrix-vector product L~_t += T_key M~_s with
//     T_key[n][m] = Dh_key[n+m] (h_s/h_t)^(|m|-s)   where |n|+|m| <= p+s, else 0.
// Targets are grouped 128 to a tile (same level and same position in the
// parent, in Morton order).  For every key that occurs in a tile, one MMA
// row block takes the sources of the 128 targets at that key as
// A [128 x n_M] (a zero row where a target has none) and T_key as
// B [n_L x n_M]:  D[128 x n_L] += A . B^T  (tcgen05.mma kind::tf32, M = 128).
// Every FP32 value is split into TF32 halves, hi + lo, and the product is
// formed as hi.hi + hi.lo + lo.hi (3xTF32) in FP32 accumulators in tensor
// memory.  The triangle |n|+|m| <= p+s is used per K-block of 8 multipoles:
// the block's MMA covers only N = (the number of n it reaches, rounded up to
// 16) columns.  Each key row is accumulated in tensor memory on its own and
// drained into FP32 registers (round to nearest); a chunk of at most G rows
// of one tile is summed there, and the chunk partials are summed in double-float
// (TwoSum pairs of floats, about 44 bits) before the final rounding to FP32.
//
// Block roles (320 threads): warps 0-7 stage A (thread = tile row and half
// of a 32-multipole K-chunk: cp.async gather into a shared ring, split,
// tcgen05.st into one of 4 tensor-memory A stages) and drain finished
// rows; lane 0 of warp 8 issues the MMAs (descriptors from a table built
// once per block) and lane 0 of warp 9 the bulk copies of the operator
// images, as far ahead as the stages allow.  A work item covers one group
// of at most W = 128 L columns: when n_L > 128 the columns from 128 on form
// a second group that needs only the first K-blocks.
//
// Each K-block takes three instructions into the row's accumulator columns
// [0, W): A_hi . B_hi^T, A_hi . B_lo^T and A_lo . B_hi^T, each N = N_kb (the
// operator image holds the hi rows, zero rows up to W, then the lo rows; a
// row's first instruction takes N = W, so its zero rows clear the columns the
// first K-block does not reach).
// Tensor memory: four row accumulators of W columns (two when W > 96), so
// that the drain of a row overlaps the MMAs of the next ones, then 2 to 4 A
// stages of hi 32 + lo 32 columns at the top.
constexpr int kTcStages = 4;
constexpr int kTcMaxAcc = 4;          // row accumulator buffers in tensor memory
constexpr int kTcThreads = 320;
constexpr int kTcMaxKB = 64;          // n_M <= 512
constexpr int kTcRawStage = 16384;    // 128 rows x 32 FP32
constexpr int kTcDrainLag = 3;        // units between a row's last staging and its drain

struct TcArgs {
    const int32_t *chunk_rb, *chunk_re;   // rows [rb, re) of each chunk
    const int32_t *row_key;               // D row of each tile row
    const int32_t *slot;                  // [rows][128] source cell, -1 = none
    const float *M;                       // scaled FP32 multipoles, row stride ldM
    const uint8_t *img;                   // per key: K-block tiles of T_key (hi, lo)
    float *partial;                       // [chunks][128][Np]
    unsigned *err;
    long long img_stride;
    int ldM, nM, n_items, ngroups, nkb, Np, b_stage_bytes;
    // row accumulators: nacc (2 or 4) buffers acc_stride columns apart; A
    // stages: nas (2..4) of 64 columns from tensor-memory column a_col0
    int nacc, acc_stride, nas, a_col0;
    // column group g covers L columns [128 g, 128 g + g_width[g]) and needs the
    // K-blocks [0, g_nkb[g]) (those that reach it), g_nkc[g] K-chunks per row
    int g_width[2], g_nkb[2], g_nkc[2];
    int kb_n[kTcMaxKB];
    int img_off[2][kTcMaxKB + 1];         // byte offset of block (g, kb) in a key image
};

// A work item is (chunk j, column group g), w = j * ngroups + g; items are
// dealt to the blocks round robin.
struct TcCursor {
    int w, j, g, r, re, kc, nkc;          // item, chunk, group, row, row end, K-chunk, K-chunks
    bool ok;
};

__device__ __forceinline__ void cur_item(TcCursor &c, const TcArgs &a)
{
    c.ok = c.w < a.n_items;
    if (!c.ok) return;
    c.j = c.w / a.ngroups;
    c.g = c.w - c.j * a.ngroups;
    c.r = a.chunk_rb[c.j];
    c.re = a.chunk_re[c.j];
    c.kc = 0;
    c.nkc = a.g_nkc[c.g];
}

__device__ __forceinline__ void cur_init(TcCursor &c, const TcArgs &a)
{
    c.w = blockIdx.x;
    cur_item(c, a);
}

__device__ __forceinline__ void cur_next(TcCursor &c, const TcArgs &a)
{
    if (!c.ok) return;
    if (++c.kc < c.nkc) return;
    c.kc = 0;
    if (++c.r < c.re) return;
    c.w += gridDim.x;
    cur_item(c, a);
}

// the row that follows the cursor's row in this block's sequence, -1 if none
__device__ __forceinline__ int cur_next_row(const TcCursor &c, const TcArgs &a)
{
    if (!c.ok) return -1;
    if (c.r + 1 < c.re) return c.r + 1;
    const int w = c.w + gridDim.x;
    return w < a.n_items ? a.chunk_rb[w / a.ngroups] : -1;
}

template <int RS>   // shared raw ring stages; RS - 1 units of A in flight
__global__ void __launch_bounds__(kTcThreads, 1) k_m2l_tc(const TcArgs a)
{
    extern __shared__ uint8_t sm_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *bst = sm;                                   // kTcStages x b_stage_bytes
    uint8_t *raw = bst + kTcStages * a.b_stage_bytes;    // RS x kTcRawStage
    uint64_t *bars = (uint64_t *)(raw + RS * kTcRawStage);
    // a_full[4] | b_full[4] | mma_done[4] | acc_empty[kTcMaxAcc]
    uint32_t *tslot = (uint32_t *)(bars + 3 * kTcStages + kTcMaxAcc);
    volatile int *abort = (volatile int *)(tslot + 1);
    // per (column group, K-block): the instruction descriptor (N = N_kb) and the
    // block's byte offset in an operator stage
    uint32_t *t_idn = (uint32_t *)(tslot + 4), *t_boff = t_idn + 2 * kTcMaxKB;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t bar0 = smem_u32(bars);
    auto a_full = [&](int i) { return bar0 + 8 * i; };
    auto b_full = [&](int i) { return bar0 + 8 * (kTcStages + i); };
    auto mma_done = [&](int i) { return bar0 + 8 * (2 * kTcStages + i); };
    auto acc_empty = [&](int i) { return bar0 + 8 * (3 * kTcStages + i); };
    if (tid == 0) {
        for (int i = 0; i < kTcStages; ++i) {
            mbar_init(a_full(i), 256);
            mbar_init(b_full(i), 1);
            mbar_init(mma_done(i), 1);
        }
        for (int i = 0; i < kTcMaxAcc; ++i) mbar_init(acc_empty(i), 256);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 8) {
        tmem_alloc(smem_u32(tslot), 512);
        tmem_relinquish();
    }
    if (warp == 9) {
        for (int e = tid - 288; e < 2 * kTcMaxKB; e += 32) {
            const int g = e / kTcMaxKB, kb = e % kTcMaxKB;
            if (g >= a.ngroups || kb >= a.g_nkb[g]) continue;
            const int c0 = 128 * g, N = min(a.kb_n[kb], c0 + 128) - c0;
            t_idn[e] = idesc_tf32_m128(N);
            t_boff[e] = (uint32_t)(a.img_off[g][kb] - a.img_off[g][kb & ~3]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp < 8) {
        // ------------------------------------------------ A producers
        const int i = tid & 127, h = tid >> 7;
        const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
        const uint32_t raw0 = smem_u32(raw) + (uint32_t)((4 * h * 128 + i) * 16);
        TcCursor cu, ci;
        cur_init(cu, a);
        ci = cu;
        int cur_row = -1, cur_src = -1, pf_row = -1, pf_src = -1;
        int ui = 0, u = 0;
        auto issue = [&]() {
            if (ci.ok) {
                if (ci.r != cur_row) {
                    cur_src = ci.r == pf_row ? pf_src : __ldg(a.slot + (size_t)ci.r * 128 + i);
                    cur_row = ci.r;
                    pf_row = cur_next_row(ci, a);
                    pf_src = pf_row >= 0 ? __ldg(a.slot + (size_t)pf_row * 128 + i) : -1;
                }
                const uint32_t dst = raw0 + (uint32_t)((ui % RS) * kTcRawStage);
                const int m0 = 32 * ci.kc + 16 * h;
                const float *row = a.M + (size_t)(cur_src < 0 ? 0 : cur_src) * a.ldM;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int m = m0 + 4 * c;
                    const int bytes = cur_src < 0 ? 0 : min(16, max(0, 4 * (a.nM - m)));
                    cp_async16(dst + c * 128 * 16, bytes ? row + m : a.M, bytes);
                }
                cur_next(ci, a);
            }
            cp_async_commit();
            ++ui;
        };
        // Each key row accumulates in its own tensor-memory buffer; once its MMAs
        // are done it is drained into FP32 registers (round to nearest), kTcDrainLag
        // units behind the staging, so that the staging does not wait for the
        // MMAs it has just enabled.  A chunk's register sum is written to
        // `partial` after its last row.  The lag stays below four units (the MMA
        // completion slots are four: a wait on a slot by parity must not see a
        // later unit's phase) and below nas + nacc units (the MMAs of a row that
        // waits for its accumulator must not hold up the staging that frees it).
        float acc[64];
#pragma unroll
        for (int c = 0; c < 64; ++c) acc[c] = 0.0f;
        int rows_seen = 0;
        TcCursor cd = cu;                            // the unit kTcDrainLag behind
        auto drain = [&](int w) -> bool {
            const bool ok = mbar_wait(mma_done(w & 3), (unsigned)((w >> 2) & 1), abort);
            if (!__all_sync(0xffffffffu, ok)) return false;
            tc_fence_after();
            const int W = a.g_width[cd.g], half = W >> 1;
            const int b = rows_seen & (a.nacc - 1);
            const uint32_t col = tmem + lane_off + (uint32_t)(b * a.acc_stride + h * half);
#pragma unroll
            for (int c = 0; c < 64; c += 32) {       // this thread's W / 2 columns, 4 loads per wait
                if (c < half) {
                    uint32_t v[32];
#pragma unroll
                    for (int q = 0; q < 32; q += 8)
                        if (c + q < half) tmem_ld8_nw(col + c + q, v + q);
#pragma unroll
                    for (int q = 0; q < 32; q += 8)
                        if (c + q < half) tmem_wait_ld8(v + q);
#pragma unroll
                    for (int k = 0; k < 32; ++k)
                        if (c + k < half) acc[c + k] += __uint_as_float(v[k]);
                }
            }
            tc_fence_before();
            mbar_arrive(acc_empty(b));
            ++rows_seen;
            if (cd.r + 1 == cd.re) {
                float *out = a.partial + ((size_t)cd.j * 128 + i) * a.Np + 128 * cd.g + h * half;
#pragma unroll
                for (int c = 0; c < 64; c += 4) {
                    if (c < half) {
                        *(float4 *)(out + c) = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
                        acc[c] = acc[c + 1] = acc[c + 2] = acc[c + 3] = 0.0f;
                    }
                }
            }
            return true;
        };
        // drain unit w if it closed a key row, then move the lagging cursor on
        auto drain_unit = [&](int w) -> bool {
            if (cd.kc == cd.nkc - 1 && !drain(w)) return false;
            cur_next(cd, a);
            return true;
        };
        const int lag = a.nacc >= 4 && a.nas >= 2 ? kTcDrainLag : 1;
        int sa = 0;                                  // A stage of unit u
        bool ok_all = true;
        for (int k = 0; k < RS - 1; ++k) issue();
        while (cu.ok) {
            issue();
            cp_async_wait<RS - 1>();
            float hi[16], lo[16];
            {
                const uint32_t src = raw0 + (uint32_t)((u % RS) * kTcRawStage);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float4 v;
                    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                                 : "r"(src + c * 128 * 16));
                    split_tf32(v.x, hi[4 * c], lo[4 * c]);
                    split_tf32(v.y, hi[4 * c + 1], lo[4 * c + 1]);
                    split_tf32(v.z, hi[4 * c + 2], lo[4 * c + 2]);
                    split_tf32(v.w, hi[4 * c + 3], lo[4 * c + 3]);
                }
            }
            // A stage sa (of nas) is free once the MMAs of unit u - nas are done
            bool ok = u < a.nas ||
                      mbar_wait_backoff(mma_done((u - a.nas) & 3), (unsigned)(((u - a.nas) >> 2) & 1), abort);
            if (!__all_sync(0xffffffffu, ok)) {
                ok_all = false;
                break;
            }
            tc_fence_after();
            const uint32_t acol = tmem + lane_off + (uint32_t)(a.a_col0 + 64 * sa + 16 * h);
            tmem_st16(acol, hi);
            tmem_st16(acol + 32, lo);
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(a_full(sa));
            if (++sa == a.nas) sa = 0;
            if (u - lag >= 0 && !drain_unit(u - lag)) {
                ok_all = false;
                break;
            }
            cur_next(cu, a);
            ++u;
        }
        // the units still to drain
        for (int w = u - lag; ok_all && w < u && !*abort; ++w)
            if (w >= 0 && !drain_unit(w)) break;
        cp_async_wait<0>();
    } else if (tid == 256) {
        // ------------------------------------------------ MMA issuer
        TcCursor cm;
        cur_init(cm, a);
        int u = 0, row_seq = 0, sa = 0, pa = 0;       // unit, key rows begun, A stage and its phase
        const uint32_t bst0 = smem_u32(bst);
        const uint64_t dconst = sdesc_sw32(0);     // descriptor bits other than the address
        const int lg = a.nacc == 4 ? 2 : (a.nacc == 2 ? 1 : 0);
        while (cm.ok) {
            const int st = u & 3;
            const bool first = cm.kc == 0;            // first unit of a key row
            const int b = row_seq & (a.nacc - 1);
            if (first && row_seq >= a.nacc &&
                !mbar_wait(acc_empty(b), (unsigned)(((row_seq >> lg) - 1) & 1), abort))
                break;
            if (!mbar_wait(a_full(sa), (unsigned)pa, abort)) break;
            if (!mbar_wait(b_full(st), (unsigned)((u >> 2) & 1), abort)) break;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(b * a.acc_stride);
            const uint32_t abase = tmem + (uint32_t)(a.a_col0 + 64 * sa);
            const uint32_t sbase = bst0 + st * a.b_stage_bytes;
            const int kb0 = 4 * cm.kc, kb1 = min(kb0 + 4, a.g_nkb[cm.g]), e0 = cm.g * kTcMaxKB;
            const uint32_t idw = idesc_tf32_m128(a.g_width[cm.g]);
            const uint32_t lo_off = 32u * (uint32_t)a.g_width[cm.g];   // the lo rows start at row W
            for (int kb = kb0; kb < kb1; ++kb) {
                const uint32_t bs = sbase + t_boff[e0 + kb];
                const uint64_t bh = dconst + (bs >> 4), bl = dconst + ((bs + lo_off) >> 4);
                const uint32_t ah = abase + 8 * (kb - kb0), al = ah + 32;
                const uint32_t idn = t_idn[e0 + kb];
                // a row's first product overwrites all W columns (the zero rows of
                // the image clear those its K-block does not reach)
                const bool clear = first && kb == kb0;
                mma_tf32_ts(d, ah, bh, clear ? idw : idn, clear ? 0u : 1u);   // hi . hi
                mma_tf32_ts(d, ah, bl, idn, 1u);                              // hi . lo
                mma_tf32_ts(d, al, bh, idn, 1u);                              // lo . hi
            }
            mma_commit(mma_done(st));
            if (cm.kc == cm.nkc - 1) ++row_seq;
            if (++sa == a.nas) {
                sa = 0;
                pa ^= 1;
            }
            cur_next(cm, a);
            ++u;
        }
        // On an abort the stagers no longer drain, so MMAs this thread issued may
        // still be running: the last commit arrives once all of them are done, and
        // tensor memory is freed below only after that (bounded) wait.
        if (*abort && u > 0) mbar_wait_cleanup(mma_done((u - 1) & 3), (unsigned)(((u - 1) >> 2) & 1));
    } else if (tid == 288) {
        // ------------------------------------------------ operator image loader
        TcCursor cb;
        cur_init(cb, a);
        int vb = 0;
        int key_row = -1, key = 0, kpf_row = -1, kpf = 0;
        const uint32_t bst0 = smem_u32(bst);
        while (cb.ok) {
            const int st = vb & 3;
            if (vb >= kTcStages && !mbar_wait(mma_done(st), (unsigned)(((vb >> 2) - 1) & 1), abort))
                break;
            if (cb.r != key_row) {
                key = cb.r == kpf_row ? kpf : __ldg(a.row_key + cb.r);
                key_row = cb.r;
                kpf_row = cur_next_row(cb, a);
                kpf = kpf_row >= 0 ? __ldg(a.row_key + kpf_row) : 0;
            }
            const int kb0 = 4 * cb.kc, kb1 = min(kb0 + 4, a.g_nkb[cb.g]);
            const unsigned bytes = (unsigned)(a.img_off[cb.g][kb1] - a.img_off[cb.g][kb0]);
            mbar_expect_tx(b_full(st), bytes);
            bulk_g2s(bst0 + st * a.b_stage_bytes, a.img + (size_t)key * a.img_stride + a.img_off[cb.g][kb0], bytes,
                     b_full(st));
            cur_next(cb, a);
            ++vb;
        }
        if (*abort) {   // let the copies still in flight land before the block exits
            for (int v = vb > kTcStages ? vb - kTcStages : 0; v < vb; ++v)
                mbar_wait_cleanup(b_full(v & 3), (unsigned)((v >> 2) & 1));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
    if (tid == 0 && *abort) atomicOr(a.err, (unsigned)kErrTcTimeout);
}

// L~_t[col_n[col]] = sum of the tile's chunk partials of target t in column col,
// in chunk order, in double-float (hi + lo FP32 pairs by TwoSum: some 44 bits,
// then rounded once to the FP32 local), a warp per target (four to a block);
// the stored components (slot r holds n = h_rn[r]: for the harmonic M2L
// exactly its columns, the n with n_z <= 1) are written, the columns no
// partial covers as zero.  NaN everywhere if a wait of the tensor-core M2L
// gave up: the failure shows in the output.
constexpr int kReduceWarps = 4;
__global__ void __launch_bounds__(32 * kReduceWarps)
k_tc_reduce(int T, const int32_t *tile_tgt, const uint32_t *tile_chunk_off, const float *partial, int Np,
            int ncol, const int32_t *col_n, int nL, int nLh, const int *h_rn, const unsigned *err, float *L)
{
    __shared__ float Ls[kReduceWarps][kMaxTot];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.x * kReduceWarps + w;
    if (q >= T) return;                   // whole warps; no block barrier below
    const bool bad = (*err & kErrTcTimeout) != 0;
    const int tile = q >> 7, tl = q & 127, c = tile_tgt[q];
    const int j0 = (int)tile_chunk_off[tile], j1 = (int)tile_chunk_off[tile + 1];
    float *ls = Ls[w];
    for (int n = lane; n < nL; n += 32) ls[n] = 0.0f;
    __syncwarp();
    for (int col = lane; col < ncol; col += 32) {
        df32 v = {0.0f, 0.0f};
        for (int j = j0; j < j1; ++j) v = df_addf(v, partial[((size_t)j * 128 + tl) * Np + col]);
        ls[col_n[col]] = __fadd_rn(v.hi, v.lo);
    }
    __syncwarp();
    for (int r = lane; r < nLh; r += 32)
        L[(size_t)c * nLh + r] = bad ? __int_as_float(0x7fc00000) : ls[h_rn[r]];
}

// ------------------------------------------------------------ the plan
// class of a target cell: (level, position in its parent); cells without
// an M2L list sort last
__global__ void k_tc_class(int64_t nc, const int32_t *m2l_off, const int32_t *level, const int32_t *cx,
                           const int32_t *cy, const int32_t *cz, uint64_t *keys, uint32_t *vals,
                           unsigned *count)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool has = false;
    if (c < nc) {
        has = m2l_off[c + 1] > m2l_off[c];
        keys[c] = has ? ((uint64_t)level[c] << 3 | (uint64_t)((cx[c] & 1) | (cy[c] & 1) << 1 | (cz[c] & 1) << 2))
                      : 0xFFFFull;
        vals[c] = (uint32_t)c;
    }
    const unsigned b = __ballot_sync(0xffffffffu, has);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(count, (unsigned)__popc(b));
}

__global__ void k_tc_tiles(int T, int slots, const uint32_t *vals, int32_t *tile_tgt)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < slots) tile_tgt[q] = q < T ? (int32_t)vals[q] : -1;
}

// The key set of each tile as a bitmap.  One block per tile: the set in
// shared memory, then written out whole (no memset, no global atomics).
constexpr int kTcBitsSmemMax = 96 * 1024;
__global__ void __launch_bounds__(256) k_tc_bits_tile(int T, const int32_t *tile_tgt, const int32_t *m2l_off,
                                                      const int32_t *didx, int W, uint32_t *bits)
{
    extern __shared__ uint32_t sb[];            // [W]
    const int tile = blockIdx.x;
    for (int i = threadIdx.x; i < W; i += blockDim.x) sb[i] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int r = threadIdx.x >> 5; r < 128; r += blockDim.x >> 5) {
        const int w = tile * 128 + r;
        if (w >= T) break;
        const int c = tile_tgt[w];
        for (int e = m2l_off[c] + lane; e < m2l_off[c + 1]; e += 32) {
            const int d = didx[e];
            atomicOr(&sb[d >> 5], 1u << (d & 31));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < W; i += blockDim.x) bits[(size_t)tile * W + i] = sb[i];
}

// The same with global atomics (one warp per target marks the keys of its
// list), for key sets too large for shared memory.
__global__ void k_tc_bits(int T, const int32_t *tile_tgt, const int32_t *m2l_off, const int32_t *didx, int W,
                          uint32_t *bits)
{
    const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= T) return;
    const int c = tile_tgt[w];
    uint32_t *tb = bits + (size_t)(w >> 7) * W;
    for (int e = m2l_off[c] + lane; e < m2l_off[c + 1]; e += 32) {
        const int d = didx[e];
        atomicOr(tb + (d >> 5), 1u << (d & 31));
    }
}

// block-wide exclusive scan of one value per thread (256 threads); returns the block total
__device__ __forceinline__ uint32_t block_scan256(uint32_t v, uint32_t &excl)
{
    __shared__ uint32_t wsum[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int k = 0; k < 8; ++k) {
        if (k < w) before += wsum[k];
        total += wsum[k];
    }
    excl = before + x - v;
    __syncthreads();
    return total;
}

// per tile: rows = keys present; prefix of the per-word counts
__global__ void __launch_bounds__(256) k_tc_rowcount(int W, int G, const uint32_t *bits, uint32_t *wpre,
                                                      uint32_t *tile_rows, uint32_t *tile_chunks)
{
    const int tile = blockIdx.x;
    uint32_t carry = 0;
    for (int base = 0; base < W; base += 256) {
        const int w = base + threadIdx.x;
        const uint32_t cnt = w < W ? (uint32_t)__popc(bits[(size_t)tile * W + w]) : 0u;
        uint32_t ex;
        const uint32_t tot = block_scan256(cnt, ex);
        if (w < W) wpre[(size_t)tile * W + w] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        tile_rows[tile] = carry;
        tile_chunks[tile] = (carry + G - 1) / G;
    }
}

__global__ void k_tc_rows(int W, int G, const uint32_t *bits, const uint32_t *wpre, const uint32_t *row_off,
                          const uint32_t *chunk_off, int32_t *row_key, int32_t *chunk_rb, int32_t *chunk_re)
{
    const int tile = blockIdx.x;
    const uint32_t rb = row_off[tile], re = row_off[tile + 1];
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        uint32_t word = bits[(size_t)tile * W + w];
        uint32_t r = rb + wpre[(size_t)tile * W + w];
        while (word) {
            const int b = __ffs(word) - 1;
            row_key[r++] = 32 * w + b;
            word &= word - 1;
        }
    }
    const int nch = (int)(chunk_off[tile + 1] - chunk_off[tile]);
    for (int k = threadIdx.x; k < nch; k += blockDim.x) {
        const int j = (int)chunk_off[tile] + k;
        chunk_rb[j] = (int32_t)(rb + (uint32_t)k * G);
        chunk_re[j] = (int32_t)min(re, rb + (uint32_t)(k + 1) * G);
    }
}

// one warp per target: place each source in its key's row, at the target's lane
__global__ void k_tc_slots(int T, const int32_t *tile_tgt, const int32_t *m2l_off, const int32_t *m2l_src,
                           const int32_t *didx, int W, const uint32_t *bits, const uint32_t *wpre,
                           const uint32_t *row_off, int32_t *slot)
{
    const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= T) return;
    const int c = tile_tgt[w], tile = w >> 7;
    const uint32_t *tb = bits + (size_t)tile * W, *tp = wpre + (size_t)tile * W;
    for (int e = m2l_off[c] + lane; e < m2l_off[c + 1]; e += 32) {
        const int d = didx[e], wd = d >> 5;
        const uint32_t r = row_off[tile] + tp[wd] + (uint32_t)__popc(tb[wd] & ((1u << (d & 31)) - 1u));
        slot[(size_t)r * 128 + (w & 127)] = m2l_src[e];
    }
}

// operator images: float e of a key's image is the hi or lo TF32 half of D
// row entry el_src[e] (or zero), at its swizzled position
__global__ void k_tc_images(int64_t ndoff, int E, const uint64_t *dkeys, const double *D, int nD,
                            const int32_t *el_src, const int32_t *el_pos, long long stride, uint8_t *img)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= ndoff * E) return;
    const int64_t r = g / E;
    const int e = (int)(g % E);
    const int src = el_src[e], pos = el_pos[e];
    float hi = 0.0f, lo = 0.0f;
    if (src >= 0) {
        const uint64_t key = dkeys[r];
        const int gap = (int)((key >> 52) & 31), tfiner = (int)((key >> 51) & 1);
        const int esc = tfiner ? 0 : gap, dl = tfiner ? gap : -gap;
        const int k = src & 0xFFFF, nm = (src >> 16) & 0xFF, msh = src >> 24;
        const double v = ldexp(D[r * nD + k], (nm + 1) * esc + dl * msh);
        hi = tf32_rna((float)v);
        lo = tf32_rna((float)(v - (double)hi));
    }
    *(float *)(img + r * stride + (pos & 0x3FFFFFFF)) = (pos >> 30) & 1 ? lo : hi;
}

}  // namespace


// ------------------------------------------------------------------ host
namespace {

inline unsigned gridn(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }
inline int up16(int n) { return std::max(16, (n + 15) & ~15); }

constexpr int kSmemMax = 232448;         // dynamic shared memory a block may opt into
constexpr int kSmemOneBlock = 120 * 1024;  // at least this much: two blocks never share an SM (and its TMEM)

int tc_smem(int b_stage, int rs)
{
    return 1024 + kTcStages * b_stage + rs * kTcRawStage + 8 * (3 * kTcStages + kTcMaxAcc) + 16 + 2 * 2 * kTcMaxKB * 4;
}

int tc_raw_stages(int b_stage)
{
    for (int rs : {8, 6, 4, 3})
        if (tc_smem(b_stage, rs) <= kSmemMax) return rs;
    return 0;
}

void build_layout(TcLayout &Ly, int s, int p, int h)
{
    const MultiIndex &I = multi_index();
    auto shell = [&](int k) { return I.nx[k] + I.ny[k] + I.nz[k]; };
    const int m0 = ntot(s - 1);
    // K runs over the kept multipoles, columns over the kept locals, both in
    // graded order (all of them, or those with z-index <= 1 when harmonic)
    std::vector<int> ms, ns;
    for (int k = m0; k < ntot(p + s); ++k)
        if (!h || I.nz[k] <= 1) ms.push_back(k);
    for (int n = 0; n < ntot(p); ++n)
        if (!h || I.nz[n] <= 1) ns.push_back(n);
    const int nM = (int)ms.size(), nL = (int)ns.size();
    Ly.s = s;
    Ly.p = p;
    Ly.h = h;
    Ly.ncol = nL;
    Ly.col_n = ns;
    Ly.nkb = (nM + 7) / 8;
    Ly.kb_n.assign(Ly.nkb, 0);
    for (int kb = 0; kb < Ly.nkb; ++kb) {  // a block's first multipole has its lowest order
        const int reach = p + s - shell(ms[8 * kb]);
        int cnt = 0;                        // the columns of order <= reach: a prefix
        while (cnt < nL && shell(ns[cnt]) <= reach) ++cnt;
        Ly.kb_n[kb] = up16(cnt);
    }
    Ly.Np = Ly.kb_n[0];
    Ly.ngroups = Ly.Np > 128 ? 2 : 1;
    Ly.img_off.assign(2 * (Ly.nkb + 1), 0);
    int off = 0;
    Ly.b_stage = 0;
    for (int g = 0; g < Ly.ngroups; ++g) {
        const int c0 = 128 * g, W = std::min(128, Ly.Np - c0);
        int nb = 0;
        while (nb < Ly.nkb && Ly.kb_n[nb] > c0) ++nb;      // reach falls with kb
        Ly.g_width[g] = W;
        Ly.g_nkb[g] = nb;
        Ly.g_nkc[g] = (nb + 3) / 4;
        int *go = &Ly.img_off[g * (Ly.nkb + 1)];
        for (int kb = 0; kb < nb; ++kb) {
            go[kb] = off;
            off += 32 * (W + std::min(Ly.kb_n[kb], c0 + 128) - c0);
        }
        for (int kb = nb; kb <= Ly.nkb; ++kb) go[kb] = off;
        for (int kc = 0; kc < Ly.g_nkc[g]; ++kc)
            Ly.b_stage = std::max(Ly.b_stage, go[std::min(4 * kc + 4, nb)] - go[4 * kc]);
    }
    Ly.img_bytes = off;
    Ly.b_stage = (Ly.b_stage + 1023) & ~1023;
    Ly.E = off / 4;
    Ly.el_src.assign(Ly.E, -1);
    Ly.el_pos.assign(Ly.E, 0);
    for (int g = 0; g < Ly.ngroups; ++g) {
        const int c0 = 128 * g, W = Ly.g_width[g];
        for (int kb = 0; kb < Ly.g_nkb[g]; ++kb) {
            const int N = std::min(Ly.kb_n[kb], c0 + 128) - c0, base = Ly.img_off[g * (Ly.nkb + 1) + kb];
            for (int row = 0; row < W + N; ++row)
                for (int k = 0; k < 8; ++k) {
                    const int pos = base + (int)swz32(row, k >> 2) + (k & 3) * 4, e = pos / 4;
                    const bool lo = row >= W;
                    Ly.el_pos[e] = pos | (lo ? 1 << 30 : 0);
                    if (row >= N && !lo) continue;               // zero rows between the halves
                    const int col = c0 + (lo ? row - W : row), m = 8 * kb + k;
                    if (m >= nM || col >= nL) continue;
                    const int n = ns[col], gm = ms[m], tot = shell(n) + shell(gm);
                    if (tot > p + s) continue;
                    const int d = I(I.nx[n] + I.nx[gm], I.ny[n] + I.ny[gm], I.nz[n] + I.nz[gm]);
                    Ly.el_src[e] = d | tot << 16 | (shell(gm) - s) << 24;
                }
        }
    }
}

fmm_status d2h_u32(fmm_tree *t, const void *dev, uint32_t *host, int count)
{
    FMM_TRY(cuda_check(t, cudaMemcpyAsync(host, dev, 4 * (size_t)count, cudaMemcpyDeviceToHost, t->stream),
                       "copy"));
    return cuda_check(t, cudaStreamSynchronize(t->stream), "sync");
}

fmm_status fail_wait(fmm_tree *t)
{
    t->err = "a bounded wait of the radix sort gave up";
    return FMM_ETIMEOUT;
}

fmm_status build_plan(fmm_tree *t)
{
    cudaStream_t st = t->stream;
    const int64_t nc = t->ncells;
    if (t->tc_G <= 0) {
        const char *g = getenv("FMM_TC_CHUNK");
        t->tc_G = g ? std::max(1, atoi(g)) : 16;
    }
    const int G = t->tc_G;
    FMM_TRY(ensure(t, t->b_tc_keys, 8 * (size_t)nc));
    FMM_TRY(ensure(t, t->b_tc_keys2, 8 * (size_t)nc));
    FMM_TRY(ensure(t, t->b_tc_vals, 4 * (size_t)nc));
    FMM_TRY(ensure(t, t->b_tc_vals2, 4 * (size_t)nc));
    const size_t hb = radix_hist_bytes(nc);
    FMM_TRY(ensure(t, t->b_tc_hist, hb));
    FMM_TRY(ensure(t, t->b_tc_scan, scan_scratch_bytes(nc + 1)));
    FMM_TRY(ensure(t, t->b_tc_cnt, 16));
    cudaMemsetAsync(t->b_tc_cnt.ptr, 0, 16, st);
    k_tc_class<<<gridn(nc, 256), 256, 0, st>>>(nc, (const int32_t *)t->b_m2l_off.ptr,
                                                (const int32_t *)t->b_level.ptr, (const int32_t *)t->b_cx.ptr,
                                                (const int32_t *)t->b_cy.ptr, (const int32_t *)t->b_cz.ptr,
                                                (uint64_t *)t->b_tc_keys.ptr, (uint32_t *)t->b_tc_vals.ptr,
                                                (unsigned *)t->b_tc_cnt.ptr);
    ++t->launches;
    radix_sort_pairs((uint64_t *)t->b_tc_keys.ptr, (uint32_t *)t->b_tc_vals.ptr, (uint64_t *)t->b_tc_keys2.ptr,
                     (uint32_t *)t->b_tc_vals2.ptr, nc, 16, (uint32_t *)t->b_tc_hist.ptr,
                     (int *)t->b_tc_cnt.ptr + 3, st, &t->launches);
    uint32_t Tw[4] = {0, 0, 0, 0};
    FMM_TRY(d2h_u32(t, t->b_tc_cnt.ptr, Tw, 4));
    if (Tw[3] & kErrSortWait) return fail_wait(t);
    const uint32_t T = Tw[0];
    t->tc_T = T;
    t->tc_tiles = (T + 127) / 128;
    t->tc_rows = t->tc_chunks = 0;
    if (T == 0) {
        t->tc_plan = true;
        return FMM_OK;
    }
    const int64_t tiles = t->tc_tiles, W = (t->n_doff + 31) / 32;
    t->tc_W = W;
    FMM_TRY(ensure(t, t->b_tc_tgt, 4 * (size_t)tiles * 128));
    k_tc_tiles<<<gridn(tiles * 128, 256), 256, 0, st>>>((int)T, (int)(tiles * 128),
                                                         (const uint32_t *)t->b_tc_vals.ptr,
                                                         (int32_t *)t->b_tc_tgt.ptr);
    FMM_TRY(ensure(t, t->b_tc_bits, 4 * (size_t)tiles * W));
    FMM_TRY(ensure(t, t->b_tc_wpre, 4 * (size_t)tiles * W));
    if (4 * W <= kTcBitsSmemMax) {
        allow_max_dynamic_smem(k_tc_bits_tile);
        k_tc_bits_tile<<<(unsigned)tiles, 256, 4 * (size_t)W, st>>>(
            (int)T, (const int32_t *)t->b_tc_tgt.ptr, (const int32_t *)t->b_m2l_off.ptr,
            (const int32_t *)t->b_m2l_didx.ptr, (int)W, (uint32_t *)t->b_tc_bits.ptr);
    } else {
        cudaMemsetAsync(t->b_tc_bits.ptr, 0, 4 * (size_t)tiles * W, st);
        k_tc_bits<<<gridn((int64_t)T * 32, 256), 256, 0, st>>>((int)T, (const int32_t *)t->b_tc_tgt.ptr,
                                                                (const int32_t *)t->b_m2l_off.ptr,
                                                                (const int32_t *)t->b_m2l_didx.ptr, (int)W,
                                                                (uint32_t *)t->b_tc_bits.ptr);
    }
    for (DevBuf *b : {&t->b_tc_rcnt, &t->b_tc_ccnt, &t->b_tc_roff, &t->b_tc_coff}) {
        FMM_TRY(ensure(t, *b, 4 * (size_t)(tiles + 1)));
        cudaMemsetAsync(b->ptr, 0, 4 * (size_t)(tiles + 1), st);
    }
    k_tc_rowcount<<<(unsigned)tiles, 256, 0, st>>>((int)W, G, (const uint32_t *)t->b_tc_bits.ptr,
                                                   (uint32_t *)t->b_tc_wpre.ptr, (uint32_t *)t->b_tc_rcnt.ptr,
                                                   (uint32_t *)t->b_tc_ccnt.ptr);
    exclusive_scan_u32((const uint32_t *)t->b_tc_rcnt.ptr, (uint32_t *)t->b_tc_roff.ptr, tiles + 1,
                       (uint32_t *)t->b_tc_scan.ptr, st, &t->launches);
    exclusive_scan_u32((const uint32_t *)t->b_tc_ccnt.ptr, (uint32_t *)t->b_tc_coff.ptr, tiles + 1,
                       (uint32_t *)t->b_tc_scan.ptr, st, &t->launches);
    t->launches += 4;
    uint32_t R = 0, C = 0;
    FMM_TRY(cuda_check(t, cudaMemcpyAsync(&R, (const uint32_t *)t->b_tc_roff.ptr + tiles, 4,
                                          cudaMemcpyDeviceToHost, st), "copy"));
    FMM_TRY(d2h_u32(t, (const uint32_t *)t->b_tc_coff.ptr + tiles, &C, 1));      // one sync for both
    t->tc_rows = R;
    t->tc_chunks = C;
    FMM_TRY(ensure(t, t->b_tc_rowkey, 4 * (size_t)R));
    FMM_TRY(ensure(t, t->b_tc_crb, 4 * (size_t)C));
    FMM_TRY(ensure(t, t->b_tc_cre, 4 * (size_t)C));
    k_tc_rows<<<(unsigned)tiles, 256, 0, st>>>((int)W, G, (const uint32_t *)t->b_tc_bits.ptr,
                                               (const uint32_t *)t->b_tc_wpre.ptr,
                                               (const uint32_t *)t->b_tc_roff.ptr,
                                               (const uint32_t *)t->b_tc_coff.ptr, (int32_t *)t->b_tc_rowkey.ptr,
                                               (int32_t *)t->b_tc_crb.ptr, (int32_t *)t->b_tc_cre.ptr);
    FMM_TRY(ensure(t, t->b_tc_slot, 4 * (size_t)R * 128));
    cudaMemsetAsync(t->b_tc_slot.ptr, 0xff, 4 * (size_t)R * 128, st);
    k_tc_slots<<<gridn((int64_t)T * 32, 256), 256, 0, st>>>(
        (int)T, (const int32_t *)t->b_tc_tgt.ptr, (const int32_t *)t->b_m2l_off.ptr,
        (const int32_t *)t->b_m2l_src.ptr, (const int32_t *)t->b_m2l_didx.ptr, (int)W,
        (const uint32_t *)t->b_tc_bits.ptr, (const uint32_t *)t->b_tc_wpre.ptr, (const uint32_t *)t->b_tc_roff.ptr,
        (int32_t *)t->b_tc_slot.ptr);
    t->launches += 2;
    t->tc_plan = true;
    return cuda_check(t, cudaGetLastError(), "tensor-core M2L plan");
}

}  // namespace

fmm_status tc_build_plan(fmm_tree *t)
{
    return build_plan(t);
}

void launch_tc_reduce(fmm_tree *t, int Np, int ncol, const int32_t *col_n, int nL, const DevTables &tb,
                      const unsigned *err, float *L)
{
    k_tc_reduce<<<(unsigned)((t->tc_T + kReduceWarps - 1) / kReduceWarps), 32 * kReduceWarps, 0, t->stream>>>(
        (int)t->tc_T, (const int32_t *)t->b_tc_tgt.ptr, (const uint32_t *)t->b_tc_coff.ptr,
        (const float *)t->b_tc_part.ptr, Np, ncol, col_n, nL, tb.nLh, tb.h_rn, err, L);
    ++t->launches;
}

bool tc_usable(fmm_tree *t, int s, int p)
{
    const int h = t->m2l_harmonic ? 1 : 0;
    if (t->tc_lay.s != s || t->tc_lay.p != p || t->tc_lay.h != h) {
        build_layout(t->tc_lay, s, p, h);
        t->tc_img_p = -1;                   // images and element maps of the old layout
    }
    const TcLayout &L = t->tc_lay;
    return L.Np <= 256 && L.nkb <= kTcMaxKB && tc_raw_stages(L.b_stage) >= 3;
}

void tc_release(fmm_tree *t)
{
    for (DevBuf *b : {&t->b_tc_keys, &t->b_tc_keys2, &t->b_tc_vals, &t->b_tc_vals2, &t->b_tc_hist,
                      &t->b_tc_scan, &t->b_tc_tgt, &t->b_tc_bits, &t->b_tc_wpre, &t->b_tc_rowkey,
                      &t->b_tc_crb, &t->b_tc_cre, &t->b_tc_slot, &t->b_tc_el, &t->b_tc_img, &t->b_tc_part,
                      &t->b_m32_el, &t->b_m32_img})
        release(t, *b);
    t->tc_plan = false;
    t->tc_img_p = -1;
    t->m32_img_p = -1;
    t->tc_T = t->tc_tiles = t->tc_rows = t->tc_chunks = 0;
}

fmm_status tc_prepare(fmm_tree *t, int p)
{
    cudaStream_t st = t->stream;
    const TcLayout &Ly = t->tc_lay;
    if (!t->tc_plan) FMM_TRY(build_plan(t));
    if (t->tc_chunks == 0) return FMM_OK;
    const long long stride = Ly.img_bytes;
    if (t->tc_img_p != p) {
        FMM_TRY(ensure(t, t->b_tc_el, 4 * (2 * (size_t)Ly.E + Ly.ncol)));
        FMM_TRY(cuda_check(t, cudaMemcpyAsync(t->b_tc_el.ptr, Ly.el_src.data(), 4 * (size_t)Ly.E,
                                              cudaMemcpyHostToDevice, st), "upload"));
        FMM_TRY(cuda_check(t, cudaMemcpyAsync((int32_t *)t->b_tc_el.ptr + Ly.E, Ly.el_pos.data(),
                                              4 * (size_t)Ly.E, cudaMemcpyHostToDevice, st), "upload"));
        FMM_TRY(cuda_check(t, cudaMemcpyAsync((int32_t *)t->b_tc_el.ptr + 2 * Ly.E, Ly.col_n.data(),
                                              4 * (size_t)Ly.ncol, cudaMemcpyHostToDevice, st), "upload"));
        FMM_TRY(ensure(t, t->b_tc_img, (size_t)t->n_doff * stride));
        k_tc_images<<<gridn(t->n_doff * Ly.E, 256), 256, 0, st>>>(
            t->n_doff, Ly.E, (const uint64_t *)t->b_dkeys.ptr, (const double *)t->b_D.ptr, ntot(p + t->s),
            (const int32_t *)t->b_tc_el.ptr, (const int32_t *)t->b_tc_el.ptr + Ly.E, stride,
            (uint8_t *)t->b_tc_img.ptr);
        ++t->launches;
        t->tc_img_p = p;
    }
    return ensure(t, t->b_tc_part, 4 * (size_t)t->tc_chunks * 128 * Ly.Np);
}

fmm_status run_m2l_tc(fmm_tree *t, int p, const float *M, int ldM, int nM, int nL,
                      const DevTables &tb, float *L)
{
    cudaStream_t st = t->stream;
    const TcLayout &Ly = t->tc_lay;
    if ((Ly.h == 1) != (tb.harmonic == 1) || nM != tb.nMh) {
        t->err = "tensor-core M2L: layout and tables disagree";
        return FMM_EINVAL;                   // not reachable: both follow the handle's flag
    }
    if (!t->tc_plan || t->tc_img_p != p) FMM_TRY(tc_prepare(t, p));
    if (t->tc_chunks == 0) return FMM_OK;
    const long long stride = Ly.img_bytes;
    if (t->tc_sms == 0) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, t->device);
        t->tc_sms = std::max(1, sms);
    }
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.chunk_rb = (const int32_t *)t->b_tc_crb.ptr;
    a.chunk_re = (const int32_t *)t->b_tc_cre.ptr;
    a.row_key = (const int32_t *)t->b_tc_rowkey.ptr;
    a.slot = (const int32_t *)t->b_tc_slot.ptr;
    a.M = M;
    a.img = (const uint8_t *)t->b_tc_img.ptr;
    a.partial = (float *)t->b_tc_part.ptr;
    unsigned *err = (unsigned *)t->b_err.ptr + 1;
    a.err = err;
    a.img_stride = stride;
    a.ldM = ldM;
    a.nM = nM;
    a.ngroups = Ly.ngroups;
    a.n_items = (int)t->tc_chunks * a.ngroups;
    a.nkb = Ly.nkb;
    a.Np = Ly.Np;
    // row accumulators of W columns (hi.hi, hi.lo and lo.hi summed in place):
    // four when they leave room for two A stages of 64 columns, else two; the
    // rest of the 512 columns hold A
    a.nacc = kTcMaxAcc * Ly.g_width[0] + 128 <= 512 ? kTcMaxAcc : 2;
    a.acc_stride = Ly.g_width[0];
    a.nas = std::min(kTcStages, (512 - a.nacc * a.acc_stride) / 64);
    a.a_col0 = 512 - 64 * a.nas;
    for (int g = 0; g < 2; ++g) {
        a.g_width[g] = Ly.g_width[g];
        a.g_nkb[g] = Ly.g_nkb[g];
        a.g_nkc[g] = Ly.g_nkc[g];
        for (int kb = 0; kb <= Ly.nkb; ++kb) a.img_off[g][kb] = Ly.img_off[g * (Ly.nkb + 1) + kb];
    }
    a.b_stage_bytes = Ly.b_stage;
    for (int kb = 0; kb < Ly.nkb; ++kb) a.kb_n[kb] = Ly.kb_n[kb];
    const int rs = tc_raw_stages(Ly.b_stage);
    const int smem = std::max(tc_smem(Ly.b_stage, rs), kSmemOneBlock);
    const unsigned grid = (unsigned)std::min<int64_t>(a.n_items, t->tc_sms);
    cudaMemsetAsync(err, 0, sizeof(unsigned), st);
    auto go = [&](auto kern) {
        allow_max_dynamic_smem(kern);
        kern<<<grid, kTcThreads, smem, st>>>(a);
    };
    switch (rs) {
    case 8: go(k_m2l_tc<8>); break;
    case 6: go(k_m2l_tc<6>); break;
    case 4: go(k_m2l_tc<4>); break;
    default: go(k_m2l_tc<3>); break;
    }
    ++t->launches;
    launch_tc_reduce(t, Ly.Np, Ly.ncol, (const int32_t *)t->b_tc_el.ptr + 2 * Ly.E, nL, tb, err, L);
    return cuda_check(t, cudaGetLastError(), "tensor-core M2L");
}

fmm_status check_umma(cudaStream_t st, const float *A, const float *B, float *D, int nkb, int N,
                      const int *kbn, int a_tmem, int passes, unsigned *err)
{
    if (nkb < 1 || nkb > 4 || N < 16 || N > 256 || N % 16 || (passes != 1 && passes != 3))
        return FMM_EINVAL;
    CheckArgs a;
    a.nkb = nkb;
    a.N = N;
    a.a_tmem = a_tmem ? 1 : 0;
    a.passes = passes;
    for (int i = 0; i < 4; ++i) a.kbn[i] = i < nkb ? kbn[i] : 16;
    if (a.kbn[0] != N) return FMM_EINVAL;
    for (int i = 0; i < nkb; ++i)
        if (a.kbn[i] < 16 || a.kbn[i] > N || a.kbn[i] % 16) return FMM_EINVAL;
    // 64 KB of slack past the tiles: every operand read stays inside the
    // block's allocation even for the widest tile a descriptor can describe
    const int smem = 1024 + 32768 + kCheckBBytes + 65536 + 64;
    allow_max_dynamic_smem(k_check_umma);
    k_check_umma<<<1, 128, smem, st>>>(A, B, D, a, err);
    return cudaGetLastError() == cudaSuccess ? FMM_OK : FMM_ECUDA;
}

}  // namespace fmm
