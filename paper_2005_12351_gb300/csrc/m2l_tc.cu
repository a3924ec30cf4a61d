// m2l_tc.cu -- the M2L translation of the FMM_3XTF32 form on the tcgen05
// tensor cores, and a self-check of the tensor-core building blocks.
#include <algorithm>
#include <cstring>

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
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

}  // namespace

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
    cudaFuncSetAttribute(k_check_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_check_umma<<<1, 128, smem, st>>>(A, B, D, a, err);
    return cudaGetLastError() == cudaSuccess ? FMM_OK : FMM_ECUDA;
}

}  // namespace fmm
