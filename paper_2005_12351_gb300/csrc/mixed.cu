// mixed.cu -- the mixed-precision form (FMM_FP32).
//
// FP64 stays where it decides accuracy: the derivative tensors of 1/r are
// generated in FP64 (one row per distinct M2L offset, shared with the FP64
// form), box-centre offsets are exact dyadic numbers, particle offsets are
// formed in FP64 before rounding, and each particle's potential and field
// are accumulated and returned in FP64.  The bulk arithmetic -- P2M, M2M,
// M2L, L2L, L2P sums and the P2P pair terms -- runs in FP32 on scaled
// expansions so that every stored value is O(1) at any tree depth.
//
// Scaling (h = half side of the cell, all factors exact powers of two):
//   M~_m = M_m / h^(|m|-s),                   L~_n = L_n h^(|n|+s+1)
//   P2M  M~_m = sum_j sum_a (-d_j)^(m-a)/(m-a)! S_{j,a},  d_j = (x_j - z)/h
//   M2M  M~p_n = 2^-(|n|-s) sum_k sig^k/k! M~c_{n-k},     sig = (z_p - z_c)/h_c
//   M2L  L~t_n += sum_m Dh_{n+m} Mh_m,  Dh_k = h_t^(|k|+1) D_k(z_t - z_s),
//        Mh_m = (h_s/h_t)^(|m|-s) M~s_m                   (Eq. (8) rescaled)
//   L2L  L~c_n += sum_k sig^k/k! 2^-(|n+k|+s+1) L~p_{n+k}, sig = (z_c - z_p)/h_c
//   L2P  phi = h^-(s+1) sum_n d^n/n! L~_n,  d_k phi = h^-(s+2) sum d^(n-e_k)/(n-e_k)! L~_n
#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "df32.cuh"
#include "fmm_internal.cuh"

namespace fmm {

namespace {

__constant__ int8_t x_nx[kMaxTot], x_ny[kMaxTot], x_nz[kMaxTot];
__constant__ float x_invint[kMaxOrder + 2];     // 1/q
__constant__ float x_invfact[kMaxOrder + 1];    // 1/q!

inline unsigned gridm(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// global row stride of the FP32 M and D tables: a multiple of 4 floats, so
// every row starts on a 16-byte boundary (rows are copied with cp.async)
__host__ __device__ __forceinline__ int row4(int n) { return (n + 3) & ~3; }


// per-axis scaled powers w^q / q!, q <= P
__device__ __forceinline__ void axis_powers32(float w, int P, float *out)
{
    float v = 1.0f;
    out[0] = 1.0f;
    for (int q = 1; q <= P; ++q) {
        v = v * w * x_invint[q];
        out[q] = v;
    }
}

// ------------------------------------------------------------------ prep
// o_j = x_j - z_leaf formed in FP64 and kept as an unevaluated float pair
// hi + lo (hi = o rounded, lo = the remainder rounded): together they carry
// ~48 bits, so pair separations can later be formed accurately relative to
// their own size.  S32 = (float)S, and after the n rows of S32 the rows of
// S32lo = (float)(S - S32), the moments' low halves for the close pairs that
// the P2P evaluates in double-float.
__device__ __forceinline__ void prep32_leaf(int c, const int32_t *begin, const int32_t *end,
                                            const double *centre, const double *px, const double *py,
                                            const double *pz, const double *S, int nS, int64_t n,
                                            float4 *o, float4 *olo, float *S32)
{
    const double z0 = centre[3 * c], z1 = centre[3 * c + 1], z2 = centre[3 * c + 2];
    const int nS32 = nS == 6 ? 7 : nS;
    float *S32lo = S32 + n * nS32;
    for (int j = begin[c] + threadIdx.x; j < end[c]; j += blockDim.x) {
        const double dx = px[j] - z0, dy = py[j] - z1, dz = pz[j] - z2;
        const float hx = (float)dx, hy = (float)dy, hz = (float)dz;
        o[j] = make_float4(hx, hy, hz, 0.0f);
        olo[j] = make_float4((float)(dx - hx), (float)(dy - hy), (float)(dz - hz), 0.0f);
        for (int a = 0; a < nS; ++a) {
            const double v = S[(int64_t)j * nS + a];
            const float vh = (float)v;
            S32[(int64_t)j * nS32 + a] = vh;
            S32lo[(int64_t)j * nS32 + a] = (float)(v - (double)vh);
        }
        if (nS == 6) {    // quadrupole trace summed in FP64: zero stays ~zero for traceless input
            const double tr = S[(int64_t)j * 6] + S[(int64_t)j * 6 + 3] + S[(int64_t)j * 6 + 5];
            const float th = (float)tr;
            S32[(int64_t)j * 7 + 6] = th;
            S32lo[(int64_t)j * 7 + 6] = (float)(tr - (double)th);
        }
    }
}

// a + b = s + e exactly (Knuth's TwoSum), then e absorbs the low part c
__device__ __forceinline__ void two_sum_lo(float a, float b, float c, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)), c);
}

// ------------------------------------------------------------------ P2M
constexpr int kChunk = 32;
constexpr int kPer = 4;                   // up to 4 * 128 = 512 components per thread block
constexpr int kMaxSrc = 6;

// One block per leaf; each thread owns up to kPer components, with the
// monomial index of each of a component's source terms taken per chunk
// (absent terms hit a zero slot).  FP32 sums over groups of 8 particles,
// double-float across groups.
__device__ __forceinline__ void p2m32_leaf(int c, const int32_t *begin, const int32_t *end,
                                           const double *half, const float4 *o, const float *S32,
                                           const DevTables &tb, float *M, float *sf)
{
    const int P = tb.p, P1 = tb.p + 1, nK = tb.nK, nK1 = tb.nK + 1, nS = tb.nS;
    float *apow = sf;                              // [chunk][3][P1]
    float *mono = apow + kChunk * 3 * P1;          // [chunk][nK + 1], last = 0
    float *Ssm = mono + kChunk * nK1;              // [chunk][8], padded with zeros
    Ssm = (float *)(((uintptr_t)Ssm + 15) & ~(uintptr_t)15);
    const int b = begin[c], e = end[c];
    // h is a power of two: 1/h from its exponent (exact, as the FP64 quotient
    // rounded to float would be), no FP64 division in every thread
    const float inv_h = ldexpf(1.0f, -ilogb(half[c]));
    const int nS32 = nS == 6 ? 7 : nS;
    df32 acc[kPer];                                // double-float: no FP64 in the pass
#pragma unroll
    for (int u = 0; u < kPer; ++u) acc[u] = {0.0f, 0.0f};
    for (int j0 = b; j0 < e; j0 += kChunk) {
        const int nj = min(kChunk, e - j0);
        for (int t = threadIdx.x; t < 3 * nj; t += blockDim.x) {
            const int j = t / 3, ax = t % 3;
            const float4 v = o[j0 + j];
            const float d = ax == 0 ? v.x : (ax == 1 ? v.y : v.z);
            axis_powers32(-d * inv_h, P, apow + (j * 3 + ax) * P1);
        }
        for (int t = threadIdx.x; t < nj * 8; t += blockDim.x)
            Ssm[t] = (t & 7) < nS ? S32[(int64_t)(j0 + (t >> 3)) * nS32 + (t & 7)] : 0.0f;
        __syncthreads();
        // each thread its monomials k (exponents decoded once) for every particle
        for (int k = threadIdx.x; k < nK1; k += blockDim.x) {
            int ox = 0, oy = 0, oz = 0;
            if (k < nK) {
                const int v = mi_at(tb.mi, k);
                ox = mi_nx(v); oy = P1 + mi_ny(v); oz = 2 * P1 + mi_nz(v);
            }
            for (int j = 0; j < nj; ++j) {
                const float *a = apow + j * 3 * P1;
                mono[j * nK1 + k] = k < nK ? a[ox] * a[oy] * a[oz] : 0.0f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int mi = threadIdx.x + u * 128;
            if (mi >= tb.nM) break;
            // the monomial index of each source term of component mi (absent: the zero slot)
            int kt[kMaxSrc];
#pragma unroll
            for (int a = 0; a < kMaxSrc; ++a) {
                const int k = a < nS ? tb.p2m_terms[mi * nS + a] : -1;
                kt[a] = k >= 0 ? k : nK;
            }
            for (int j8 = 0; j8 < nj; j8 += 8) {
                float sum = 0.0f;
                const int je = min(j8 + 8, nj);
                for (int j = j8; j < je; ++j) {
                    const float *mj = mono + j * nK1;
                    const float4 s0 = *(const float4 *)(Ssm + 8 * j);
                    sum = fmaf(mj[kt[0]], s0.x, sum);
                    if (nS > 1) sum = fmaf(mj[kt[1]], s0.y, sum);
                    if (nS > 2) sum = fmaf(mj[kt[2]], s0.z, sum);
                    if (nS > 3) sum = fmaf(mj[kt[3]], s0.w, sum);
                    if (nS > 4) {
                        const float2 s1 = *(const float2 *)(Ssm + 8 * j + 4);
                        sum = fmaf(mj[kt[4]], s1.x, sum);
                        if (nS > 5) sum = fmaf(mj[kt[5]], s1.y, sum);
                    }
                }
                acc[u] = df_addf(acc[u], sum);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int mi = threadIdx.x + u * 128;
        if (mi < tb.nM) M[(int64_t)c * row4(tb.nM) + mi] = __fadd_rn(acc[u].hi, acc[u].lo);
    }
}

// sig^k / k! with sig_d = +1 or -1 given by neg_d (1 means -1)
__device__ __forceinline__ float sign_mono(const int *mi, int k, int nx_neg, int ny_neg, int nz_neg)
{
    const int v = mi_at(mi, k);
    const int kx = mi_nx(v), ky = mi_ny(v), kz = mi_nz(v);
    const int odd = (nx_neg & kx) ^ (ny_neg & ky) ^ (nz_neg & kz);
    const float m = x_invfact[kx] * x_invfact[ky] * x_invfact[kz];
    return (odd & 1) ? -m : m;
}

// ------------------------------------------------------------------ M2M
// parent c from its children (the rows may have been written by other blocks
// of the same launch: ldcg).  The children's sign-monomial tables and rows are
// staged together, so the block meets once, not twice per child.
__device__ __forceinline__ void m2m32_cell(int c, const int32_t *child, const int32_t *nchild,
                                           const int32_t *cx, const int32_t *cy, const int32_t *cz,
                                           const DevTables &tb, float *M, float *sf)
{
    const int nch = nchild[c], nK = tb.nK, nM = tb.nM;
    float *mono = sf;               // [nch][nK]
    float *Mc = mono + 8 * nK;      // [nch][nM]
    for (int i = 0; i < nch; ++i) {
        const int ch = child[c] + i;
        // z_p - z_c = (1 - 2 bit) h_c per axis: negative where the child's low bit is 1
        const int bx = cx[ch] & 1, by = cy[ch] & 1, bz = cz[ch] & 1;
        for (int k = threadIdx.x; k < nK; k += blockDim.x) mono[i * nK + k] = sign_mono(tb.mi, k, bx, by, bz);
        for (int t = threadIdx.x; t < nM; t += blockDim.x) Mc[i * nM + t] = __ldcg(M + (int64_t)ch * row4(nM) + t);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int ni = threadIdx.x + u * 128;
        if (ni >= nM) break;
        const int q0 = tb.m2m_off[ni], q1 = tb.m2m_off[ni + 1];
        df32 acc = {0.0f, 0.0f};
        for (int i = 0; i < nch; ++i) {
            const float *mo = mono + i * nK, *mc = Mc + i * nM;
            float sum = 0.0f;
            for (int q = q0; q < q1; ++q) sum = fmaf(mo[tb.m2m_k[q]], mc[tb.m2m_q[q]], sum);
            acc = df_addf(acc, sum);
        }
        const int sc = -(mi_shell(mi_at(tb.mi, ni + tb.m0)) - tb.s);     // a power of two: exact
        M[(int64_t)c * row4(nM) + ni] = ldexpf(__fadd_rn(acc.hi, acc.lo), sc);
    }
}

// The upward pass of this form in one launch: the float offsets and moments
// of leaf b's particles (prep32_leaf), its P2M, then the block whose child
// arrives last at a parent forms the parent's multipole, up to the root (the
// FP64 form's k_upward, same counters and ordering).
__global__ void __launch_bounds__(128, 8)
k_upward32(const int32_t *leaves, const int32_t *begin, const int32_t *end, const int32_t *parent,
           const int32_t *child, const int32_t *nchild, const int32_t *cx, const int32_t *cy,
           const int32_t *cz, const double *half, const double *centre, const double *px,
           const double *py, const double *pz, const double *S, int nS_in, int64_t n, float4 *o,
           float *S32, DevTables tb, float *M, unsigned *arrive)
{
    extern __shared__ float sf[];
    __shared__ int s_go;
    int c = leaves[blockIdx.x];
    prep32_leaf(c, begin, end, centre, px, py, pz, S, nS_in, n, o, o + n, S32);
    __syncthreads();
    p2m32_leaf(c, begin, end, half, o, S32, tb, M, sf);
    for (;;) {
        const int pa = parent[c];
        if (pa < 0) break;
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned n = atomicAdd(&arrive[pa], 1u) + 1u;
            const bool last = n == (unsigned)nchild[pa];
            if (last) {
                arrive[pa] = 0u;
                __threadfence();
            }
            s_go = last;
        }
        __syncthreads();
        if (!s_go) break;
        m2m32_cell(pa, child, nchild, cx, cy, cz, tb, M, sf);
        c = pa;
    }
}

// ------------------------------------------------------------ D rows, FP32
// Dh_k = h_t^(|k|+1) D_k(u v) = (h_t/u)^(|k|+1) D_k(v): the unit-free FP64 row
// shifted by the level gap when the target is the coarser cell (h_t = 2^gap u),
// unchanged otherwise (h_t = u), and rounded once.
__global__ void k_dtables32(const uint64_t *dkeys, int64_t ndoff, int nD, const double *D,
                            const int *mi, float *D32)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ndoff * nD) return;
    const int64_t r = i / nD;
    const int k = (int)(i % nD);
    const uint64_t key = dkeys[r];
    const int gap = (int)((key >> 52) & 31), tfiner = (int)((key >> 51) & 1);
    const int e = tfiner ? 0 : gap;
    D32[r * row4(nD) + k] = (float)ldexp(D[i], (mi_shell(mi_at(mi, k)) + 1) * e);
}

// ------------------------------------------------------------------ M2L
constexpr int kM2LThreads = 128;
constexpr int kBatch = 16;

__global__ void __launch_bounds__(kM2LThreads)
k_m2l32(const int32_t *off, const int32_t *src, const int32_t *didx, const int32_t *level,
        const float *M, const float *D32, DevTables tb, float *L)
{
    extern __shared__ float sf[];
    const int c = blockIdx.x;
    const int b = off[c], e = off[c + 1];
    if (b == e) return;
    // M: the kept (folded, when harmonic) scaled multipole rows, row4(nMh) per cell
    const int nM = tb.nMh, nD = tb.nD, T = tb.m2l_T, Tn = kM2LThreads;
    const int ldM = nM | 1, ldD = nD | 1;
    double *part = (double *)sf;                   // [slots][Tn], FP64 across batches
    float *Msm = (float *)(part + tb.m2l_slots * Tn);   // [batch][ldM]
    float *Dsm = Msm + kBatch * ldM;               // [batch][ldD]
    uint32_t *desc = (uint32_t *)(Dsm + kBatch * ldD);  // [T][Tn]
    const int tid = threadIdx.x;
    const int lt = level[c];
    __shared__ int bsrc[kBatch], bdidx[kBatch], bdl[kBatch];
    for (int i = tid; i < T * Tn; i += Tn) desc[i] = tb.m2l_desc[i];
    for (int i = tid; i < tb.m2l_slots * Tn; i += Tn) part[i] = 0.0;
    for (int k0 = b; k0 < e; k0 += kBatch) {
        const int kb = min(kBatch, e - k0);
        __syncthreads();
        if (tid < kb) {                    // batch metadata, loaded in parallel
            const int s = src[k0 + tid];
            bsrc[tid] = s;
            bdidx[tid] = didx[k0 + tid];
            bdl[tid] = lt - level[s];
        }
        __syncthreads();
        for (int k = 0; k < kb; ++k) {
            const float *Ms = M + (int64_t)bsrc[k] * row4(nM);
            const int dl = bdl[k];
            for (int m = tid; m < nM; m += Tn) {
                float v = Ms[m];
                if (dl) v = ldexpf(v, dl * (mi_shell(mi_at(tb.mi, tb.h_rm[m] + tb.m0)) - tb.s));
                Msm[k * ldM + m] = v;
            }
            const float *Dk = D32 + (int64_t)bdidx[k] * row4(nD);
            for (int d = tid; d < nD; d += Tn) Dsm[k * ldD + d] = Dk[d];
        }
        __syncthreads();
        float acc = 0.0f;
        for (int t = 0; t < T; ++t) {
            const uint32_t u = desc[t * Tn + tid];
            if (u == 0xffffffffu) break;
            const float *Mp = Msm + (u & 511u);
            const float *Dp = Dsm + ((u >> 9) & 511u);
            int k = 0;
            for (; k + 4 <= kb; k += 4) {
                acc = fmaf(Dp[k * ldD], Mp[k * ldM], acc);
                acc = fmaf(Dp[(k + 1) * ldD], Mp[(k + 1) * ldM], acc);
                acc = fmaf(Dp[(k + 2) * ldD], Mp[(k + 2) * ldM], acc);
                acc = fmaf(Dp[(k + 3) * ldD], Mp[(k + 3) * ldM], acc);
            }
            for (; k < kb; ++k) acc = fmaf(Dp[k * ldD], Mp[k * ldM], acc);
            if (u & (1u << 18)) {
                part[(u >> 19) * Tn + tid] += (double)acc;
                acc = 0.0f;
            }
        }
    }
    __syncthreads();
    // the stored components (n_z <= 1 when harmonic, the traceless form)
    for (int r = tid; r < tb.nLh; r += Tn) {
        const int n = tb.h_rn[r];
        double v = 0.0;
        for (int q = tb.m2l_red_off[n]; q < tb.m2l_red_off[n + 1]; ++q) v += part[tb.m2l_red_src[q]];
        L[(int64_t)c * tb.nLh + r] = (float)v;
    }
}

// ------------------------------------------------------------------ L2L
__device__ __forceinline__ void l2l32_cell(int c, int pa, const int32_t *cx, const int32_t *cy,
                                           const int32_t *cz, const DevTables &tb, float *L, float *sf)
{
    float *mono = sf;               // [nK]
    float *Lp = mono + tb.nK;       // [nL], pre-scaled by 2^-(|q|+s+1)
    // z_c - z_p = (2 bit - 1) h_c: negative where the child's low bit is 0
    const int bx = 1 - (cx[c] & 1), by = 1 - (cy[c] & 1), bz = 1 - (cz[c] & 1);
    for (int k = threadIdx.x; k < tb.nK; k += blockDim.x) mono[k] = sign_mono(tb.mi, k, bx, by, bz);
    // the parent's full expansion (the identity holds degree by degree, so the
    // power-of-two rescaling may follow the unfold)
    expand_local_cg(L + (int64_t)pa * tb.nLh, tb, Lp);
    for (int q = threadIdx.x; q < tb.nL; q += blockDim.x)
        Lp[q] = ldexpf(Lp[q], -(mi_shell(mi_at(tb.mi, q)) + tb.s + 1));
    __syncthreads();
    for (int r = threadIdx.x; r < tb.nLh; r += blockDim.x) {
        const int n = tb.h_rn[r];
        if (mi_shell(mi_at(tb.mi, n)) < tb.n_lo) continue;
        float acc = 0.0f;
        for (int q = tb.l2l_off[n]; q < tb.l2l_off[n + 1]; ++q)
            acc = fmaf(mono[tb.l2l_k[q]], Lp[tb.l2l_q[q]], acc);
        L[(int64_t)c * tb.nLh + r] += acc;
    }
}

// ------------------------------------------------------------------ L2P
constexpr int kL2PThreads = 128;

// L2P of leaf c by one block of kL2PThreads (shared memory sf: n_L +
// kL2PThreads x 3 (p + 1) floats).  A leaf holds fewer particles than the
// block has threads, so tp = a power of two of thread groups shares the
// particles (the largest with tp x count <= the block): thread (slice sl,
// particle jl) sums every tp-th term of particle jl.  The slices run across
// warps, so a warp's lanes read the same term tables (constant-cache
// broadcast), and the tp partial sums meet in shared memory in slice order.
// CG: L was written earlier in the same launch (read through L2).
template <bool CG>
__device__ __forceinline__ void l2p32_leaf(int c, const int32_t *begin, const int32_t *end, const double *half,
                                           const float4 *o, const float *L, const DevTables &tb, int want_phi,
                                           int want_field, double *phi, double *E, float *sf)
{
    __shared__ float part[4][kL2PThreads];
    const int P = tb.p, P1 = tb.p + 1;
    float *Lsm = sf;                                       // [nL]
    float *apow = Lsm + tb.nL;                             // [particles of a chunk][3][P1]
    const int b = begin[c], e = end[c], nt = e - b;
    const double h = half[c];
    const int eh = ilogb(h);
    const float inv_h = ldexpf(1.0f, -eh);                 // h = 2^eh: exact, no FP64 division
    const double sphi = ldexp(1.0, -(tb.s + 1) * eh), sfield = ldexp(1.0, -(tb.s + 2) * eh);
    int tp = 1;
    while (tp < 32 && 2 * tp * nt <= kL2PThreads) tp *= 2;
    const int npc = kL2PThreads / tp;
    const int jl = threadIdx.x % npc, sl = threadIdx.x / npc;
    expand_local<float, CG>(L + (int64_t)c * tb.nLh, tb, Lsm);
    for (int j0 = b; j0 < e; j0 += npc) {
        const int j = j0 + jl;
        const bool act = j < e;
        float *a = apow + jl * 3 * P1;
        if (act)
            for (int ax = sl; ax < 3; ax += tp) {
                const float4 v = o[j];
                axis_powers32((ax == 0 ? v.x : (ax == 1 ? v.y : v.z)) * inv_h, P, a + ax * P1);
            }
        __syncthreads();
        float f = 0.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
        if (act && want_phi)
            for (int k = sl; k < tb.nL; k += tp)
                f = fmaf(a[x_nx[k]] * a[P1 + x_ny[k]] * a[2 * P1 + x_nz[k]], Lsm[k], f);
        if (act && want_field)
            for (int k = sl; k < tb.nG; k += tp) {
                const float m = a[x_nx[k]] * a[P1 + x_ny[k]] * a[2 * P1 + x_nz[k]];
                g0 = fmaf(m, Lsm[tb.l2p_grad[3 * k]], g0);
                g1 = fmaf(m, Lsm[tb.l2p_grad[3 * k + 1]], g1);
                g2 = fmaf(m, Lsm[tb.l2p_grad[3 * k + 2]], g2);
            }
        part[0][threadIdx.x] = f; part[1][threadIdx.x] = g0;
        part[2][threadIdx.x] = g1; part[3][threadIdx.x] = g2;
        __syncthreads();
        if (act && sl == 0) {
            for (int u = 1; u < tp; ++u) {
                f += part[0][u * npc + jl]; g0 += part[1][u * npc + jl];
                g1 += part[2][u * npc + jl]; g2 += part[3][u * npc + jl];
            }
            if (want_phi) phi[j] = (double)f * sphi;
            if (want_field) {
                E[3 * (int64_t)j] = -(double)g0 * sfield;
                E[3 * (int64_t)j + 1] = -(double)g1 * sfield;
                E[3 * (int64_t)j + 2] = -(double)g2 * sfield;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kL2PThreads)
k_l2p32(const int32_t *leaves, const int32_t *begin, const int32_t *end, const double *half,
        const float4 *o, const float *L, DevTables tb, int want_phi, int want_field,
        double *phi, double *E)
{
    extern __shared__ float sf[];
    l2p32_leaf<false>(leaves[blockIdx.x], begin, end, half, o, L, tb, want_phi, want_field, phi, E, sf);
}

// The L2L shifts of this form in two launches.  First the cells with
// children, in breadth-first order (as the FP64 form's k_downward: a block
// claims the next one through a counter, waits, bounded, for its parent's
// flag, shifts, publishes; NaN where a wait gave up); inner = those cells in
// index order.  Then the leaves, whose parents are final: each block shifts
// its leaf and runs its L2P, with no claim and no wait (the leaves are most
// of the cells, and one counter claimed by every block serialises them).
__global__ void __launch_bounds__(128)
k_downward32(int64_t nint, const int32_t *inner, const int32_t *parent, const int32_t *cx,
             const int32_t *cy, const int32_t *cz, DevTables tb, float *L, unsigned *ctl)
{
    extern __shared__ float sf[];
    __shared__ int s_k, s_ok;
    if (threadIdx.x == 0) s_k = (int)atomicAdd(&ctl[0], 1u);
    __syncthreads();
    if (s_k >= nint) return;
    const int c = inner[s_k];
    const int pa = parent[c];
    if (pa >= 0) {
        if (threadIdx.x == 0) {
            s_ok = wait_flag(ctl + 1 + pa);
            __threadfence();
        }
        __syncthreads();
        if (s_ok) {
            l2l32_cell(c, pa, cx, cy, cz, tb, L, sf);
        } else {
            for (int r = threadIdx.x; r < tb.nLh; r += blockDim.x)
                L[(int64_t)c * tb.nLh + r] = __int_as_float(0x7fc00000);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicExch(ctl + 1 + c, 1u);
    }
}

__global__ void __launch_bounds__(128)
k_downward32_leaf(const int32_t *leaves, const int32_t *parent, const int32_t *cx, const int32_t *cy,
                  const int32_t *cz, DevTables tb, float *L, const int32_t *begin, const int32_t *end,
                  const double *half, const float4 *o, int want_phi, int want_field, double *phi, double *E)
{
    extern __shared__ float sf[];
    const int c = leaves[blockIdx.x], pa = parent[c];
    if (pa >= 0) {
        l2l32_cell(c, pa, cx, cy, cz, tb, L, sf);
        __syncthreads();                 // the leaf's expansion is final: its L2P reads it back
    }
    l2p32_leaf<true>(c, begin, end, half, o, L, tb, want_phi, want_field, phi, E, sf);
}

// ------------------------------------------------------------------ P2P
// FP32 pair terms on coordinates relative to the target leaf's centre:
// target o_i, source o_j + (z_B - z_A), the centre offset formed exactly from
// the integer cell coordinates.  Each thread sums a staged round in FP32 and
// adds it to double-float totals, the copies' totals meet in double-float,
// and the far field is added in FP64.
//
// Close pairs.  A target's field error in FP32 pair arithmetic is set by its
// nearest neighbours (the pair terms grow as r^-(s+2) and the rounding of
// each is relative to its own size), so the pairs closer than one mean
// particle spacing of the target leaf, a = 2 h / count^(1/3), are evaluated in
// double-float arithmetic instead (df32.cuh; ~4 pairs per particle in a
// uniform set, ~0.2 % of the near field), which puts the near field's
// rounding at the level of the FP64 form.  The FP32 loop zeroes such a pair
// and queues it for its thread and target; when a queue of the warp is full,
// and at the end of each staged round, the warp's queued pairs are dealt to
// all its lanes, evaluated, and added by their owners to their double-float
// sums in queue order, so the result stays deterministic.  Only the sources
// staged near the target leaf (first in a round's order) can make close
// pairs; the far ones run a step without the test.
// the hardware reciprocal square root (PTX rsqrt.approx, relative error ~2^-23);
// callers pass normal x > 0 only
__device__ __forceinline__ float rsqrt_mufu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// keep = false: the pair contributes nothing (a close pair, evaluated in
// double-float instead, or r = 0)
template <int S, bool PHI, bool FIELD>
__device__ __forceinline__ void pair32(float dx, float dy, float dz, float r2, bool keep, const float *Sj,
                                       float &f, float &e0, float &e1, float &e2)
{
    float y = keep ? rsqrt_mufu(r2) : 0.0f;
    y = y * fmaf(-0.5f * r2 * y, y, 1.5f);          // one Newton step: ~1 ulp
    const float y2 = y * y;
    if (S == 0) {
        if (PHI) f = fmaf(Sj[0], y, f);
        if (FIELD) {
            const float w = Sj[0] * (y * y2);
            e0 = fmaf(w, dx, e0); e1 = fmaf(w, dy, e1); e2 = fmaf(w, dz, e2);
        }
    } else if (S == 1) {
        const float y3 = y * y2;
        const float sr = fmaf(Sj[0], dx, fmaf(Sj[1], dy, Sj[2] * dz));
        if (PHI) f = fmaf(-sr, y3, f);
        if (FIELD) {
            const float w = 3.0f * sr * (y3 * y2);
            e0 = fmaf(Sj[0], y3, fmaf(-w, dx, e0));
            e1 = fmaf(Sj[1], y3, fmaf(-w, dy, e1));
            e2 = fmaf(Sj[2], y3, fmaf(-w, dz, e2));
        }
    } else {
        const float y3 = y * y2, y5 = y3 * y2;
        const float gq0 = fmaf(2.0f * Sj[0], dx, fmaf(Sj[1], dy, Sj[2] * dz));
        const float gq1 = fmaf(Sj[1], dx, fmaf(2.0f * Sj[3], dy, Sj[4] * dz));
        const float gq2 = fmaf(Sj[2], dx, fmaf(Sj[4], dy, 2.0f * Sj[5] * dz));
        const float q = 0.5f * fmaf(gq0, dx, fmaf(gq1, dy, gq2 * dz));
        const float tr = Sj[6];
        if (PHI) f += 3.0f * q * y5 - tr * y3;
        if (FIELD) {
            const float a = 3.0f * y5;
            const float w = fmaf(15.0f * q, y5 * y2, -3.0f * tr * y5);
            e0 = fmaf(w, dx, fmaf(-a, gq0, e0));
            e1 = fmaf(w, dy, fmaf(-a, gq1, e1));
            e2 = fmaf(w, dz, fmaf(-a, gq2, e2));
        }
    }
}

// Two FP32 lanes in one 64-bit register (low half = first): the f32x2
// arithmetic of sm_100 and later, each half rounded as the scalar operation
// would be, one issue slot for both.
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_pack(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(f2 v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// a constant in both halves, formed in plain integer arithmetic (foldable and
// hoistable, unlike a pack through inline assembly)
__device__ __forceinline__ f2 f2_splat(float a)
{
    const f2 u = (f2)__float_as_uint(a);
    return u | (u << 32);
}

// pair32 for two targets at once (one per half), the same operations in the
// same order, so that each half's sums are those of pair32; y comes in as
// the two seeds (0 where the pair is not kept).  Sj holds each source term
// twice, as pairs.
template <int S, bool PHI, bool FIELD>
__device__ __forceinline__ void pair32x2(f2 dx, f2 dy, f2 dz, f2 r2, f2 y, const f2 *Sj, f2 &f, f2 &e0,
                                         f2 &e1, f2 &e2)
{
    y = f2_mul(y, f2_fma(f2_mul(f2_mul(f2_splat(-0.5f), r2), y), y, f2_splat(1.5f)));
    const f2 y2 = f2_mul(y, y);
    if (S == 0) {
        if (PHI) f = f2_fma(Sj[0], y, f);
        if (FIELD) {
            const f2 w = f2_mul(Sj[0], f2_mul(y, y2));
            e0 = f2_fma(w, dx, e0); e1 = f2_fma(w, dy, e1); e2 = f2_fma(w, dz, e2);
        }
    } else if (S == 1) {
        const f2 y3 = f2_mul(y, y2);
        const f2 sr = f2_fma(Sj[0], dx, f2_fma(Sj[1], dy, f2_mul(Sj[2], dz)));
        if (PHI) f = f2_fma(f2_mul(sr, f2_splat(-1.0f)), y3, f);
        if (FIELD) {
            const f2 nw = f2_mul(f2_mul(f2_splat(-3.0f), sr), f2_mul(y3, y2));   // -w exactly
            e0 = f2_fma(Sj[0], y3, f2_fma(nw, dx, e0));
            e1 = f2_fma(Sj[1], y3, f2_fma(nw, dy, e1));
            e2 = f2_fma(Sj[2], y3, f2_fma(nw, dz, e2));
        }
    } else {
        const f2 y3 = f2_mul(y, y2), y5 = f2_mul(y3, y2);
        const f2 two = f2_splat(2.0f);
        const f2 gq0 = f2_fma(f2_mul(two, Sj[0]), dx, f2_fma(Sj[1], dy, f2_mul(Sj[2], dz)));
        const f2 gq1 = f2_fma(Sj[1], dx, f2_fma(f2_mul(two, Sj[3]), dy, f2_mul(Sj[4], dz)));
        const f2 gq2 = f2_fma(Sj[2], dx, f2_fma(Sj[4], dy, f2_mul(f2_mul(two, Sj[5]), dz)));
        const f2 q = f2_mul(f2_splat(0.5f), f2_fma(gq0, dx, f2_fma(gq1, dy, f2_mul(gq2, dz))));
        const f2 tr = Sj[6];
        if (PHI) f = f2_add(f, f2_fma(f2_mul(f2_splat(3.0f), q), y5, f2_mul(f2_mul(tr, y3), f2_splat(-1.0f))));
        if (FIELD) {
            const f2 na = f2_mul(f2_splat(-3.0f), y5);
            const f2 w = f2_fma(f2_mul(f2_splat(15.0f), q), f2_mul(y5, y2),
                                f2_mul(f2_mul(f2_splat(-3.0f), tr), y5));
            e0 = f2_fma(w, dx, f2_fma(na, gq0, e0));
            e1 = f2_fma(w, dy, f2_fma(na, gq1, e1));
            e2 = f2_fma(w, dz, f2_fma(na, gq2, e2));
        }
    }
}

// the same separation as a double-float: (oi - a) by TwoSum, the low parts added
__device__ __forceinline__ df32 sep_df(float oi, float li, float a, float b)
{
    const df32 d = df_two_sum(oi, -a);
    return df_fast2(d.hi, __fadd_rn(d.lo, __fsub_rn(li, b)));
}

constexpr int kP2PThreads = 128;
constexpr int kGroups = 64;
constexpr int kLaneQ = 8;                 // close pairs a thread queues per target
constexpr double kCloseSpacings = 1.0;    // close: r < this many mean spacings of the target leaf

// TT: targets per thread (1 or 2; the autotuner's tile choice): two share each
// staged source read, one leaves more threads per target and fewer registers.
template <int S, bool PHI, bool FIELD, int TT>
__global__ void __launch_bounds__(kP2PThreads, S == 2 ? 4 : 6)
k_p2p32(const int32_t *leaves, const int32_t *begin, const int32_t *end, const int32_t *off,
        const int32_t *src, const int32_t *level, const int32_t *cx, const int32_t *cy,
        const int32_t *cz, const int32_t *sys, const double *sys_box, const double *half,
        const float4 *o, const float4 *olo, const float *S32, const float *S32lo,
        const double *phi_far, const double *E_far, const int32_t *perm, double *phi_out,
        double *E_out)
{
    constexpr int nS = S == 2 ? 7 : (S + 1) * (S + 2) / 2;     // + trace for quadrupoles
    constexpr int nR2 = (nS - 1 + 1) / 2;                       // float4s of moments after the first
    constexpr int CH = S == 2 ? 448 : (S == 1 ? 512 : 688);   // 6 blocks per SM for S < 2
    // a round stages at most CHU sources; the slots up to CH take the padding
    // that gives every thread the same number of steps
    constexpr int CHU = CH - kP2PThreads;
    // staged sources of a round, every value twice (the f32x2 pairs of the
    // two-target step): PD = (x, x, y, y), QD = (z, z, S_0, S_0) hi position in
    // the target leaf's frame and first moment, RD = the other moments two to a
    // float4, then the positions' low parts; the per-thread totals of the final
    // reduction reuse the same bytes once the last round is done
    constexpr int kStageFloats = CH * (8 + 4 * nR2 + 3);
    static_assert(kStageFloats >= 2 * 8 * kP2PThreads, "reduction area");
    __shared__ __align__(16) float stage[kStageFloats];
    float4 *PD = (float4 *)stage, *QD = PD + CH, *RD = QD + CH;
    float *lx = (float *)(RD + nR2 * CH), *ly = lx + CH, *lz = ly + CH;
    df32 (*red)[kP2PThreads] = (df32 (*)[kP2PThreads])stage;
    __shared__ int gbeg[kGroups], gpre[kGroups + 1];
    __shared__ float gdx[kGroups], gdy[kGroups], gdz[kGroups];
    __shared__ int s_next_q, s_next_j, s_ngroups;
    // per thread and target: staged indices of its queued close pairs
    __shared__ uint16_t closeq[2][kLaneQ][kP2PThreads];
    // a round's slots in pair-loop order: the sources near the target leaf first
    __shared__ uint16_t order[CH];
    __shared__ int s_wnear[kP2PThreads / 32];
    const int c = leaves[blockIdx.x];
    const int b = begin[c], e = end[c], nt = e - b;
    const int q0 = off[c], q1 = off[c + 1];
    const int tid = threadIdx.x;
    const int lc = level[c];
    const long long rc = 1ll << (kLevels - lc);
    const long long ccx = (2ll * cx[c] + 1) * rc, ccy = (2ll * cy[c] + 1) * rc,
                    ccz = (2ll * cz[c] + 1) * rc;
    const double unit = ldexp(sys_box[4 * sys[c] + 3], -(kLevels + 1));   // finest half-cell
    // squared close-pair radius of this leaf's targets (FP64 cube root: formed
    // once per block, not per thread)
    __shared__ float s_close2;
    if (tid == 0) {
        const double sp_a = kCloseSpacings * 2.0 * half[c] / cbrt((double)max(nt, 1));
        s_close2 = (float)(sp_a * sp_a);
    }
    __syncthreads();
    const float close2 = s_close2;
    // a source is near when its squared distance to the leaf's box is under
    // the close radius squared with a 2 % margin: only near sources can make a
    // close pair (far ones are beyond the radius from every target, well past
    // the FP32 rounding of the separations)
    const float hw = (float)half[c], near2 = 1.02f * close2;
    for (int t0 = 0; t0 < nt; t0 += TT * kP2PThreads) {
        const int cnt = min(TT * kP2PThreads, nt - t0);
        const int h = TT == 2 ? (cnt + 1) / 2 : cnt;
        const int k = max(1, kP2PThreads / h);
        const int ti = tid % h, sp = tid / h;
        const bool act = sp < k;
        const bool two = TT == 2 && act && (ti + h < cnt);
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 oi = act ? o[b + t0 + ti] : zero4;
        const float4 oj = two ? o[b + t0 + ti + h] : oi;
        // totals of the tile in double-float: the rounds' FP32 sums and the
        // close pairs both go in
        df32 cF[2] = {{0.f, 0.f}, {0.f, 0.f}}, cA[2] = {{0.f, 0.f}, {0.f, 0.f}};
        df32 cB[2] = {{0.f, 0.f}, {0.f, 0.f}}, cC[2] = {{0.f, 0.f}, {0.f, 0.f}};
        int qa = 0, qb = 0;                          // close pairs queued for each target
        // Evaluate this thread's queued close pairs in double-float into its own
        // sums, in queue order; the lanes of a warp work side by side.
        // Evaluate the warp's queued close pairs in double-float: the queues of
        // all lanes (each lane's target-0 entries, then its target-1 entries)
        // are dealt to the lanes 32 at a time, each lane evaluating one pair
        // into zeroed sums; then every owner adds its pairs' results to its own
        // sums in queue order, so the result is that of evaluating them in turn.
        auto flush = [&]() {
            const unsigned full = 0xffffffffu;
            const int lane = tid & 31, wtid = tid - lane;
            __syncwarp();
            const int myn = qa + qb;
            int incl = myn;
#pragma unroll
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
                const int y = __shfl_up_sync(full, incl, o2);
                if (lane >= o2) incl += y;
            }
            const int tot = __shfl_sync(full, incl, 31), excl = incl - myn;
            for (int c0 = 0; c0 < tot; c0 += 32) {
                const int e = c0 + lane;
                // the entry's owner: the first lane whose inclusive count exceeds e
                int L = 0;
#pragma unroll
                for (int st = 16; st > 0; st >>= 1) {
                    const int v = __shfl_sync(full, incl, L + st - 1);
                    if (v <= e) L += st;
                }
                L = min(L, 31);
                const int oqa = __shfl_sync(full, qa, L), oex = __shfl_sync(full, excl, L);
                df32 rf = {0.f, 0.f}, r0 = {0.f, 0.f}, r1 = {0.f, 0.f}, r2 = {0.f, 0.f};
                if (e < tot) {
                    const int t = e - oex, w = t < oqa ? 0 : 1, u = w ? t - oqa : t;
                    const int otid = wtid + L;
                    const int d = closeq[w][u][otid];
                    const int ot = otid % h + w * h;         // the owner's target in the tile
                    const float4 po = o[b + t0 + ot], pl = olo[b + t0 + ot];
                    // the staged source's particle index: its group by the prefix of sizes
                    int lo = 0, hi = s_ngroups - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (gpre[mid] <= d) lo = mid; else hi = mid - 1;
                    }
                    const int64_t jsrc = gbeg[lo] + (d - gpre[lo]);
                    float sl[nS], sh[nS];
                    const float4 pd = PD[d], qd = QD[d];
                    sh[0] = qd.z;
#pragma unroll
                    for (int a2 = 1; a2 < nS; ++a2) {
                        const float4 r = RD[d * nR2 + (a2 - 1) / 2];
                        sh[a2] = (a2 - 1) % 2 ? r.z : r.x;
                    }
#pragma unroll
                    for (int a2 = 0; a2 < nS; ++a2) sl[a2] = S32lo[jsrc * nS + a2];
                    pair_df<S, PHI, FIELD>(sep_df(po.x, pl.x, pd.x, lx[d]), sep_df(po.y, pl.y, pd.z, ly[d]),
                                           sep_df(po.z, pl.z, qd.x, lz[d]), sh, sl, rf, r0, r1, r2);
                }
                // my own entries in this batch of 32: positions [s0, s1)
                const int s0 = max(excl - c0, 0), s1 = min(incl - c0, 32);
                const int cnt_max = (int)__reduce_max_sync(full, (unsigned)max(s1 - s0, 0));
                for (int jj = 0; jj < cnt_max; ++jj) {
                    const int srcl = min(s0 + jj, 31);
                    const df32 vf = {__shfl_sync(full, rf.hi, srcl), __shfl_sync(full, rf.lo, srcl)};
                    const df32 v0 = {__shfl_sync(full, r0.hi, srcl), __shfl_sync(full, r0.lo, srcl)};
                    const df32 v1 = {__shfl_sync(full, r1.hi, srcl), __shfl_sync(full, r1.lo, srcl)};
                    const df32 v2 = {__shfl_sync(full, r2.hi, srcl), __shfl_sync(full, r2.lo, srcl)};
                    if (s0 + jj < s1) {
                        const int te = c0 + s0 + jj - excl;      // my entry index
                        if (te < qa) {
                            if (PHI) cF[0] = df_add(cF[0], vf);
                            if (FIELD) { cA[0] = df_add(cA[0], v0); cB[0] = df_add(cB[0], v1); cC[0] = df_add(cC[0], v2); }
                        } else if constexpr (TT == 2) {
                            if (PHI) cF[1] = df_add(cF[1], vf);
                            if (FIELD) { cA[1] = df_add(cA[1], v0); cB[1] = df_add(cB[1], v1); cC[1] = df_add(cC[1], v2); }
                        }
                    }
                }
            }
            __syncwarp();
            qa = qb = 0;
        };
        int q = q0, j_in = 0;
        while (q < q1) {
            __syncthreads();
            if (tid < 32) {
                // warp 0 takes up to 32 partner leaves of this round in parallel: lane l
                // the entry q + l (the first continues at j_in); a prefix sum of their
                // sizes decides which fit in CHU (the last one possibly in part)
                const int lane = tid;
                const int qq = q + lane;
                int lb = 0, take = 0, sl = 0;
                if (qq < q1) {
                    sl = src[qq];
                    lb = begin[sl] + (lane == 0 ? j_in : 0);
                    take = end[sl] - lb;
                }
                int incl = take;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int excl = incl - take;
                const bool in = qq < q1 && excl < CHU;
                const int tk = in ? min(take, CHU - excl) : 0;
                if (in) {
                    const long long rs = 1ll << (kLevels - level[sl]);
                    gbeg[lane] = lb;
                    gpre[lane] = excl;
                    gdx[lane] = (float)((double)((2ll * cx[sl] + 1) * rs - ccx) * unit);
                    gdy[lane] = (float)((double)((2ll * cy[sl] + 1) * rs - ccy) * unit);
                    gdz[lane] = (float)((double)((2ll * cz[sl] + 1) * rs - ccz) * unit);
                }
                const int ng = __popc(__ballot_sync(0xffffffffu, in));   // the taken entries: a prefix
                if (lane == ng - 1) {
                    const bool whole = tk == take;
                    gpre[ng] = excl + tk;
                    s_ngroups = ng;
                    s_next_q = whole ? qq + 1 : qq;
                    s_next_j = whole ? 0 : (lb - begin[sl]) + tk;
                }
            }
            __syncthreads();
            const int ng = s_ngroups, used = gpre[ng];
            // every thread takes the same number of steps (the close-pair
            // evaluation between stretches of them is warp-collective)
            const int steps = (used + k - 1) / k;
            uint32_t nbits = 0;                // bit i: slot tid + 128 i is near
            int nmine = 0;
            for (int d = tid, i = 0; d < steps * k; d += kP2PThreads, ++i) {
                if (d >= used) {
                    // padding: a far-away source with zero moments adds exactly 0
                    PD[d] = make_float4(1e18f, 1e18f, 1e18f, 1e18f);
                    QD[d] = make_float4(1e18f, 1e18f, 0.0f, 0.0f);
#pragma unroll
                    for (int a = 0; a < nR2; ++a) RD[d * nR2 + a] = make_float4(0.f, 0.f, 0.f, 0.f);
                    lx[d] = ly[d] = lz[d] = 0.0f;
                    continue;
                }
                int lo = 0, hi = ng - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (gpre[mid] <= d) lo = mid; else hi = mid - 1;
                }
                const int j = gbeg[lo] + (d - gpre[lo]);
                const float4 v = o[j], vl = olo[j];
                // source position in the target leaf's frame, as an exact hi + lo pair
                float hx, hy, hz;
                two_sum_lo(v.x, gdx[lo], vl.x, hx, lx[d]);
                two_sum_lo(v.y, gdy[lo], vl.y, hy, ly[d]);
                two_sum_lo(v.z, gdz[lo], vl.z, hz, lz[d]);
                const float s0 = S32[(int64_t)j * nS];
                PD[d] = make_float4(hx, hx, hy, hy);
                QD[d] = make_float4(hz, hz, s0, s0);
#pragma unroll
                for (int a = 0; a < nR2; ++a) {
                    const float u = S32[(int64_t)j * nS + 2 * a + 1];
                    const float v = 2 * a + 2 < nS ? S32[(int64_t)j * nS + 2 * a + 2] : 0.0f;
                    RD[d * nR2 + a] = make_float4(u, u, v, v);
                }
                const float bx = fmaxf(fabsf(hx) - hw, 0.0f), by = fmaxf(fabsf(hy) - hw, 0.0f),
                            bz = fmaxf(fabsf(hz) - hw, 0.0f);
                if (bx * bx + by * by + bz * bz < near2) {
                    nbits |= 1u << i;
                    ++nmine;
                }
            }
            // the loop order: near slots first (ranked by thread, then slot),
            // then the far ones and the padding
            int n_near;
            {
                const int lane = tid & 31, w = tid >> 5;
                int incl = nmine;
#pragma unroll
                for (int o2 = 1; o2 < 32; o2 <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o2);
                    if (lane >= o2) incl += y;
                }
                if (lane == 31) s_wnear[w] = incl;
                __syncthreads();
                int base = 0;
                n_near = 0;
#pragma unroll
                for (int u = 0; u < kP2PThreads / 32; ++u) {
                    if (u < w) base += s_wnear[u];
                    n_near += s_wnear[u];
                }
                const int S_ = steps * k, full = S_ / kP2PThreads, rem = S_ % kP2PThreads;
                int rn = base + incl - nmine;                       // near slots of the threads before
                int rf = n_near + tid * full + min(tid, rem) - rn;  // far slots of the threads before
                for (int d = tid, i = 0; d < S_; d += kP2PThreads, ++i)
                    order[(nbits >> i) & 1u ? rn++ : rf++] = (uint16_t)d;
            }
            __syncthreads();
            const int steps_near = (n_near + k - 1) / k;
            // The pair loop only queues close pairs; they are evaluated when a
            // queue of the warp is full and after the round.  Threads without a
            // target (and the second target of a thread that has one only) run
            // the loop on a copy with a zero close radius; their sums are never read.
            const int spx = act ? sp : 0;
            const float c2a = act ? close2 : 0.0f, c2b = two ? close2 : 0.0f;
            // sums of the round: (target a, target b) pairs
            f2 Fp = 0ull, E0p = 0ull, E1p = 0ull, E2p = 0ull;
            const f2 OX = f2_pack(oi.x, oj.x), OY = f2_pack(oi.y, oj.y), OZ = f2_pack(oi.z, oj.z);
            // one step: source slot spx + it k against the thread's targets
            float f1 = 0.f, e10 = 0.f, e11 = 0.f, e12 = 0.f;    // one target per thread: scalar sums
            // NEAR: the slot may hold a near source (close-pair test and queue)
            auto step = [&](int it2, auto near_t) {
                constexpr bool NEAR = decltype(near_t)::value;
                const int jj = order[spx + it2 * k];
                if constexpr (TT == 1) {
                    const float4 pd = PD[jj], qd = QD[jj];
                    float Sj[nS];
                    Sj[0] = qd.z;
#pragma unroll
                    for (int a = 0; a < nR2; ++a) {
                        const float4 r = RD[jj * nR2 + a];
                        Sj[2 * a + 1] = r.x;
                        if (2 * a + 2 < nS) Sj[2 * a + 2] = r.z;
                    }
                    const float dx = oi.x - pd.x, dy = oi.y - pd.z, dz = oi.z - qd.x;
                    const float r2a = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    pair32<S, PHI, FIELD>(dx, dy, dz, r2a, !NEAR || r2a >= c2a, Sj, f1, e10, e11, e12);
                    if (NEAR && r2a < c2a && r2a > 0.0f) closeq[0][qa++][tid] = (uint16_t)jj;
                    return;
                }
                const ulonglong2 pd = reinterpret_cast<const ulonglong2 *>(PD)[jj];
                const ulonglong2 qd = reinterpret_cast<const ulonglong2 *>(QD)[jj];
                f2 Sj[nS];
                Sj[0] = qd.y;
#pragma unroll
                for (int a = 0; a < nR2; ++a) {
                    const ulonglong2 r = reinterpret_cast<const ulonglong2 *>(RD)[jj * nR2 + a];
                    Sj[2 * a + 1] = r.x;
                    if (2 * a + 2 < nS) Sj[2 * a + 2] = r.y;
                }
                // separations from the rounded leaf-frame coordinates: the error is
                // ~1 ulp of the leaf size, small next to r for every pair this
                // loop keeps (the closer ones go to the double-float queue, which
                // takes the low parts too)
                const f2 dx = f2_sub(OX, pd.x), dy = f2_sub(OY, pd.y), dz = f2_sub(OZ, qd.x);
                const f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
                const float2 r2s = f2_unpack(r2);
                if constexpr (!NEAR) {
                    // every pair is kept: beyond the close radius, r > 0
                    pair32x2<S, PHI, FIELD>(dx, dy, dz, r2, f2_pack(rsqrt_mufu(r2s.x), rsqrt_mufu(r2s.y)), Sj,
                                            Fp, E0p, E1p, E2p);
                    return;
                }
                const bool ka = r2s.x >= c2a, kb = r2s.y >= c2b;
                const f2 y = f2_pack(ka ? rsqrt_mufu(r2s.x) : 0.0f, (TT == 2 && kb) ? rsqrt_mufu(r2s.y) : 0.0f);
                pair32x2<S, PHI, FIELD>(dx, dy, dz, r2, y, Sj, Fp, E0p, E1p, E2p);
                if (r2s.x < c2a && r2s.x > 0.0f) closeq[0][qa++][tid] = (uint16_t)jj;
                if (TT == 2 && r2s.y < c2b && r2s.y > 0.0f) closeq[1][qb++][tid] = (uint16_t)jj;
            };
            const std::integral_constant<bool, true> near_s;
            const std::integral_constant<bool, false> far_s;
            int it = 0;
            while (it < steps_near) {
                // two steps, then a look at the queues: they have room for two more
                bool full = false;
                for (; it + 1 < steps_near; it += 2) {
                    step(it, near_s);
                    step(it + 1, near_s);
                    if (__any_sync(0xffffffffu, qa > kLaneQ - 2 || qb > kLaneQ - 2)) {
                        it += 2;
                        full = true;
                        break;
                    }
                }
                if (!full && it < steps_near) step(it++, near_s);    // an odd last step
                if (__any_sync(0xffffffffu, qa + qb > 0)) flush();   // staged sources change next round
            }
            // the far slots: no close pairs, nothing queued
#pragma unroll 4
            for (; it < steps; ++it) step(it, far_s);
            {
                if constexpr (TT == 1) {
                    cF[0] = df_addf(cF[0], f1); cA[0] = df_addf(cA[0], e10);
                    cB[0] = df_addf(cB[0], e11); cC[0] = df_addf(cC[0], e12);
                } else {
                    const float2 f = f2_unpack(Fp), e0 = f2_unpack(E0p), e1 = f2_unpack(E1p), e2 = f2_unpack(E2p);
                    cF[0] = df_addf(cF[0], f.x); cA[0] = df_addf(cA[0], e0.x);
                    cB[0] = df_addf(cB[0], e1.x); cC[0] = df_addf(cC[0], e2.x);
                    cF[1] = df_addf(cF[1], f.y); cA[1] = df_addf(cA[1], e0.y);
                    cB[1] = df_addf(cB[1], e1.y); cC[1] = df_addf(cC[1], e2.y);
                }
            }
            q = s_next_q;
            j_in = s_next_j;
        }
        __syncthreads();
        // the k copies' totals meet in double-float (no FP64 until the far field joins)
        red[0][tid] = cF[0]; red[1][tid] = cA[0]; red[2][tid] = cB[0]; red[3][tid] = cC[0];
        red[4][tid] = cF[1]; red[5][tid] = cA[1]; red[6][tid] = cB[1]; red[7][tid] = cC[1];
        __syncthreads();
        if (tid < h) {
#pragma unroll
            for (int half = 0; half < TT; ++half) {
                if (half == 1 && tid + h >= cnt) break;
                const int r = 4 * half;
                df32 Fv = red[r][tid], Av = red[r + 1][tid], Bv = red[r + 2][tid], Cv = red[r + 3][tid];
                for (int u = 1; u < k; ++u) {
                    Fv = df_add(Fv, red[r][u * h + tid]);
                    Av = df_add(Av, red[r + 1][u * h + tid]);
                    Bv = df_add(Bv, red[r + 2][u * h + tid]);
                    Cv = df_add(Cv, red[r + 3][u * h + tid]);
                }
                const int ii = b + t0 + tid + half * h;
                const int64_t oo = perm[ii];
                if (PHI) phi_out[oo] = phi_far[ii] + df_to_double(Fv);
                if (FIELD) {
                    E_out[3 * oo] = E_far[3 * (int64_t)ii] + df_to_double(Av);
                    E_out[3 * oo + 1] = E_far[3 * (int64_t)ii + 1] + df_to_double(Bv);
                    E_out[3 * oo + 2] = E_far[3 * (int64_t)ii + 2] + df_to_double(Cv);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------- symmetric P2P
// The near field by Newton's third law in this form's FP32 pair arithmetic,
// on the plan of the FP64 symmetric P2P (mirror entries, reverse rows): each
// mirrored leaf pair (A, B) with B > A is evaluated once by A's block, in A's
// frame (source positions taken there by the exact hi + lo sum); the forward
// terms of a target are summed over the warp in FP32 and across warps in
// FP64, the reverse terms of a source over A's targets in FP32 into its row,
// which the gather adds in FP64 in list order.  The reverse term is the
// forward formula with the target's moments and -R (parity (-1)^s for the
// potential of an order-s source, (-1)^(s+1) for its field).
constexpr int kSym32Threads = 128;
constexpr int kSym32Warps = kSym32Threads / 32;
constexpr int kSym32Targets = 128;

// moment terms a pair reads: S, or for quadrupoles (2 S200, S110, S101, 2 S020,
// S011, 2 S002, trace) from the S32 row (S, trace)
template <int S> struct Sym32Mom { static constexpr int n = S == 2 ? 7 : (S + 1) * (S + 2) / 2; };

template <int S>
__device__ __forceinline__ void sym32_load_mom(const float *Sj, float *m)
{
    if (S < 2) {
#pragma unroll
        for (int a = 0; a < (S + 1) * (S + 2) / 2; ++a) m[a] = Sj[a];
    } else {
        m[0] = 2.0f * Sj[0]; m[1] = Sj[1]; m[2] = Sj[2]; m[3] = 2.0f * Sj[3]; m[4] = Sj[4];
        m[5] = 2.0f * Sj[5]; m[6] = Sj[6];
    }
}

struct Sym32Geo {
    float dx, dy, dz, y, y3, c1, c2, c3;
};

template <int S, bool PHI, bool FIELD>
__device__ __forceinline__ Sym32Geo sym32_geo(float dx, float dy, float dz)
{
    Sym32Geo g;
    g.dx = dx; g.dy = dy; g.dz = dz;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float y = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
    y = y * fmaf(-0.5f * r2 * y, y, 1.5f);          // one Newton step, as pair32
    const float y2 = y * y;
    g.y = y;
    g.y3 = y * y2;
    g.c1 = g.c2 = g.c3 = 0.0f;
    if (S == 1 && FIELD) g.c1 = 3.0f * y2;
    if (S == 2) {
        const float y5 = g.y3 * y2;
        g.c1 = 3.0f * y5;
        if (PHI) g.c2 = 1.5f * y5;
        if (FIELD) g.c3 = 7.5f * (y5 * y2);
    }
    return g;
}

// one direction into a = ([phi], [E]): forward (source moments m) or, with REV,
// reverse (the target's moments, R -> -R)
template <int S, bool PHI, bool FIELD, bool REV>
__device__ __forceinline__ void sym32_dir(const Sym32Geo &g, const float *m, float *a)
{
    constexpr int e = PHI ? 1 : 0;
    if (S == 0) {
        if (PHI) a[0] = fmaf(m[0], g.y, a[0]);
        if (FIELD) {
            const float w = REV ? -(m[0] * g.y3) : m[0] * g.y3;
            a[e] = fmaf(w, g.dx, a[e]);
            a[e + 1] = fmaf(w, g.dy, a[e + 1]);
            a[e + 2] = fmaf(w, g.dz, a[e + 2]);
        }
    } else if (S == 1) {
        const float sr = fmaf(m[0], g.dx, fmaf(m[1], g.dy, m[2] * g.dz));
        if (PHI) a[0] = fmaf(REV ? sr : -sr, g.y3, a[0]);
        if (FIELD) {
            const float v = sr * g.c1;
            a[e] = fmaf(fmaf(-v, g.dx, m[0]), g.y3, a[e]);
            a[e + 1] = fmaf(fmaf(-v, g.dy, m[1]), g.y3, a[e + 1]);
            a[e + 2] = fmaf(fmaf(-v, g.dz, m[2]), g.y3, a[e + 2]);
        }
    } else {
        const float gq0 = fmaf(m[0], g.dx, fmaf(m[1], g.dy, m[2] * g.dz));
        const float gq1 = fmaf(m[1], g.dx, fmaf(m[3], g.dy, m[4] * g.dz));
        const float gq2 = fmaf(m[2], g.dx, fmaf(m[4], g.dy, m[5] * g.dz));
        const float q2 = fmaf(gq0, g.dx, fmaf(gq1, g.dy, gq2 * g.dz));   // 2 q(R)
        const float tr = m[6];
        if (PHI) a[0] = fmaf(q2, g.c2, fmaf(-tr, g.y3, a[0]));
        if (FIELD) {
            const float w = fmaf(q2, g.c3, -tr * g.c1);
            const float wa = REV ? -w : w, ca = REV ? g.c1 : -g.c1;
            a[e] = fmaf(wa, g.dx, fmaf(ca, gq0, a[e]));
            a[e + 1] = fmaf(wa, g.dy, fmaf(ca, gq1, a[e + 1]));
            a[e + 2] = fmaf(wa, g.dz, fmaf(ca, gq2, a[e + 2]));
        }
    }
}

// warp totals of four partial sums, fixed pattern: lanes 8c .. 8c+7 hold v_c's
__device__ __forceinline__ float sym32_warp_sum4(float v0, float v1, float v2, float v3)
{
    const int lane = threadIdx.x & 31;
    const bool h16 = lane & 16, h8 = lane & 8;
    float a = h16 ? v2 : v0, b = h16 ? v3 : v1;
    const float sa = h16 ? v0 : v2, sb = h16 ? v1 : v3;
    a += __shfl_xor_sync(0xffffffffu, sa, 16);
    b += __shfl_xor_sync(0xffffffffu, sb, 16);
    float c = h8 ? b : a;
    const float sc = h8 ? a : b;
    c += __shfl_xor_sync(0xffffffffu, sc, 8);
    c += __shfl_xor_sync(0xffffffffu, c, 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

__device__ __forceinline__ float sym32_warp_sum1(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// one batch of sources (d0 + u * kSym32Threads + tid, u < TJ) against the
// staged targets; with REV the reverse terms go to the sources' rows
template <int S, bool PHI, bool FIELD, bool REV, int TJ>
__device__ __forceinline__ void sym32_batch(int d0, int used, int ne, const int *seg_q, const int *seg_pre,
                                            const float *seg_dx, const float *seg_dy, const float *seg_dz,
                                            const int32_t *src, const int32_t *begin, const uint32_t *rbase,
                                            const float4 *o, const float4 *olo, const float *S32,
                                            const float *tx, const float *ty, const float *tz,
                                            const float *ux, const float *uy, const float *uz,
                                            const float *tm, int cntT, float (*fw)[4], float *rev, bool first)
{
    constexpr int nS = S == 2 ? 7 : (S + 1) * (S + 2) / 2;
    constexpr int nM = Sym32Mom<S>::n;
    constexpr int NC = (PHI ? 1 : 0) + (FIELD ? 3 : 0);
    const int tid = threadIdx.x, lane = tid & 31;
    float sx[TJ], sy[TJ], sz[TJ], lx[TJ], ly[TJ], lz[TJ], sm[TJ][nM], acc[TJ][NC];
    int64_t row[TJ];
    bool val[TJ];
#pragma unroll
    for (int u = 0; u < TJ; ++u) {
        const int d = d0 + u * kSym32Threads + tid;
        val[u] = d < used;
        sx[u] = sy[u] = sz[u] = lx[u] = ly[u] = lz[u] = 0.0f;
#pragma unroll
        for (int a = 0; a < nM; ++a) sm[u][a] = 0.0f;
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[u][c] = 0.0f;
        row[u] = 0;
        if (val[u]) {
            int lo = 0, hi = ne - 1;          // last entry with seg_pre <= d
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (seg_pre[mid] <= d) lo = mid; else hi = mid - 1;
            }
            const int q = seg_q[lo], k = d - seg_pre[lo];
            const int j = begin[src[q]] + k;
            const float4 v = o[j], vl = olo[j];
            two_sum_lo(v.x, seg_dx[lo], vl.x, sx[u], lx[u]);
            two_sum_lo(v.y, seg_dy[lo], vl.y, sy[u], ly[u]);
            two_sum_lo(v.z, seg_dz[lo], vl.z, sz[u], lz[u]);
            sym32_load_mom<S>(S32 + (int64_t)j * nS, sm[u]);
            if (REV) row[u] = (int64_t)rbase[q] + k;
        }
    }
    for (int i = 0; i < cntT; ++i) {
        const float xi = tx[i], yi = ty[i], zi = tz[i], xl = ux[i], yl = uy[i], zl = uz[i];
        float mi[nM];
#pragma unroll
        for (int a = 0; a < nM; ++a) mi[a] = REV ? tm[i * nM + a] : 0.0f;
        float f[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int u = 0; u < TJ; ++u) {
            if (!val[u]) continue;
            // hi parts of nearby points subtract exactly; the lo parts restore the rest
            const Sym32Geo g = sym32_geo<S, PHI, FIELD>((xi - sx[u]) + (xl - lx[u]), (yi - sy[u]) + (yl - ly[u]),
                                                        (zi - sz[u]) + (zl - lz[u]));
            sym32_dir<S, PHI, FIELD, false>(g, sm[u], f);
            if (REV) sym32_dir<S, PHI, FIELD, true>(g, mi, acc[u]);
        }
        if (NC == 1) {
            const float v = sym32_warp_sum1(f[0]);
            if (lane == 0) fw[i][0] += v;
        } else {
            const float v = sym32_warp_sum4(f[0], f[1], f[2], NC == 4 ? f[3] : 0.0f);
            if ((lane & 7) == 0 && (lane >> 3) < NC) fw[i][lane >> 3] += v;
        }
    }
    if (REV) {
#pragma unroll
        for (int u = 0; u < TJ; ++u) {
            if (!val[u]) continue;
            float *r = rev + row[u] * NC;
#pragma unroll
            for (int c = 0; c < NC; ++c) r[c] = first ? acc[u][c] : r[c] + acc[u][c];
        }
    }
}

// One block per target leaf A, rounds of up to kSym32Targets staged targets;
// pass 0: mirrored entries with B > A (both directions), pass 1: the
// forward-only entries (A itself, entries without a mirror); A's row walked in
// segments of 32 entries compacted by warp 0.
template <int S, bool PHI, bool FIELD>
__global__ void __launch_bounds__(kSym32Threads)
k_p2p32_sym(const int32_t *leaves, const int32_t *begin, const int32_t *end, const int32_t *off,
            const int32_t *src, const int32_t *mir, const uint32_t *rbase, const int32_t *level,
            const int32_t *cx, const int32_t *cy, const int32_t *cz, const int32_t *sys,
            const double *sys_box, const float4 *o, const float4 *olo, const float *S32, float *rev,
            double *fwd)
{
    constexpr int nS = S == 2 ? 7 : (S + 1) * (S + 2) / 2;
    constexpr int nM = Sym32Mom<S>::n;
    constexpr int NC = (PHI ? 1 : 0) + (FIELD ? 3 : 0);
    constexpr int TJ = 4;
    __shared__ float tx[kSym32Targets], ty[kSym32Targets], tz[kSym32Targets];
    __shared__ float ux[kSym32Targets], uy[kSym32Targets], uz[kSym32Targets], tm[kSym32Targets * nM];
    __shared__ float fw[kSym32Warps][kSym32Targets][4];
    __shared__ int seg_q[32], seg_pre[33];
    __shared__ float seg_dx[32], seg_dy[32], seg_dz[32];
    __shared__ int s_ne;
    const int A = leaves[blockIdx.x];
    const int b = begin[A], nA = end[A] - b;
    const int q0 = off[A], q1 = off[A + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long rc = 1ll << (kLevels - level[A]);
    const long long ccx = (2ll * cx[A] + 1) * rc, ccy = (2ll * cy[A] + 1) * rc, ccz = (2ll * cz[A] + 1) * rc;
    const double unit = ldexp(sys_box[4 * sys[A] + 3], -(kLevels + 1));   // finest half-cell
    for (int t0 = 0; t0 == 0 || t0 < nA; t0 += kSym32Targets) {
        const int cntT = max(0, min(kSym32Targets, nA - t0));
        __syncthreads();
        for (int u = tid; u < cntT; u += kSym32Threads) {
            const int i = b + t0 + u;
            const float4 v = o[i], vl = olo[i];
            tx[u] = v.x; ty[u] = v.y; tz[u] = v.z;
            ux[u] = vl.x; uy[u] = vl.y; uz[u] = vl.z;
            sym32_load_mom<S>(S32 + (int64_t)i * nS, tm + u * nM);
        }
        for (int u = tid; u < kSym32Warps * kSym32Targets * 4; u += kSym32Threads) (&fw[0][0][0])[u] = 0.0f;
        for (int pass = 0; pass < 2; ++pass) {
            for (int qs = q0; qs < q1; qs += 32) {
                __syncthreads();
                if (warp == 0) {
                    const int q = qs + lane;
                    int n = 0, take = 0, B = 0;
                    if (q < q1) {
                        B = src[q];
                        const int m = mir[q];
                        take = pass == 0 ? (m >= 0 && B > A) : (B == A || m < 0);
                        if (take) n = end[B] - begin[B];
                    }
                    int k = take, c = n;
#pragma unroll
                    for (int o2 = 1; o2 < 32; o2 <<= 1) {
                        const int yk = __shfl_up_sync(0xffffffffu, k, o2);
                        const int yc = __shfl_up_sync(0xffffffffu, c, o2);
                        if (lane >= o2) { k += yk; c += yc; }
                    }
                    if (take) {
                        const long long rs = 1ll << (kLevels - level[B]);
                        seg_q[k - 1] = q;
                        seg_pre[k - 1] = c - n;
                        seg_dx[k - 1] = (float)((double)((2ll * cx[B] + 1) * rs - ccx) * unit);
                        seg_dy[k - 1] = (float)((double)((2ll * cy[B] + 1) * rs - ccy) * unit);
                        seg_dz[k - 1] = (float)((double)((2ll * cz[B] + 1) * rs - ccz) * unit);
                    }
                    if (lane == 31) { s_ne = k; seg_pre[k] = c; }
                }
                __syncthreads();
                const int ne = s_ne, used = seg_pre[ne];
                for (int d0 = 0; d0 < used; d0 += kSym32Threads * TJ) {
                    if (pass == 0)
                        sym32_batch<S, PHI, FIELD, true, TJ>(d0, used, ne, seg_q, seg_pre, seg_dx, seg_dy, seg_dz,
                                                             src, begin, rbase, o, olo, S32, tx, ty, tz, ux, uy,
                                                             uz, tm, cntT, fw[warp], rev, t0 == 0);
                    else
                        sym32_batch<S, PHI, FIELD, false, TJ>(d0, used, ne, seg_q, seg_pre, seg_dx, seg_dy,
                                                              seg_dz, src, begin, rbase, o, olo, S32, tx, ty,
                                                              tz, ux, uy, uz, tm, cntT, fw[warp], rev, false);
                }
            }
        }
        __syncthreads();
        for (int u = tid; u < cntT; u += kSym32Threads) {
            const int64_t i = b + t0 + u;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                double v = (double)fw[0][u][c];
#pragma unroll
                for (int w = 1; w < kSym32Warps; ++w) v += (double)fw[w][u][c];
                fwd[i * NC + c] = v;
            }
        }
    }
}

// per target of leaf A: the forward sum, the reverse rows of each mirrored
// entry (A, B) with B < A in list order (FP64), then the far field
template <bool PHI, bool FIELD>
__global__ void __launch_bounds__(kSym32Threads)
k_p2p32_sym_gather(const int32_t *leaves, const int32_t *begin, const int32_t *end, const int32_t *off,
                   const int32_t *src, const int32_t *mir, const uint32_t *rbase, const float *rev,
                   const double *fwd, const double *phi_far, const double *E_far, const int32_t *perm,
                   double *phi_out, double *E_out)
{
    constexpr int NC = (PHI ? 1 : 0) + (FIELD ? 3 : 0);
    constexpr int e = PHI ? 1 : 0;
    const int A = leaves[blockIdx.x];
    const int b = begin[A], nA = end[A] - b;
    const int q0 = off[A], q1 = off[A + 1];
    for (int u = threadIdx.x; u < nA; u += kSym32Threads) {
        const int64_t i = b + u;
        double v[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = fwd[i * NC + c];
        for (int q = q0; q < q1; ++q) {
            const int B = src[q], m = mir[q];
            if (m < 0 || B >= A) continue;
            const float *r = rev + ((int64_t)rbase[m] + u) * NC;
#pragma unroll
            for (int c = 0; c < NC; ++c) v[c] += (double)r[c];
        }
        const int64_t oo = perm[i];
        if (PHI) phi_out[oo] = phi_far[i] + v[0];
        if (FIELD) {
            E_out[3 * oo] = E_far[3 * i] + v[e];
            E_out[3 * oo + 1] = E_far[3 * i + 1] + v[e + 1];
            E_out[3 * oo + 2] = E_far[3 * i + 2] + v[e + 2];
        }
    }
}

template <int S>
void launch_p2p32_sym(fmm_tree *t, int want_phi, int want_field, double *phi, double *E)
{
    const unsigned g = (unsigned)t->nleaves;
    cudaStream_t st = t->stream;
    const int32_t *lv = (const int32_t *)t->b_leaves.ptr, *bg = (const int32_t *)t->b_begin.ptr,
                  *en = (const int32_t *)t->b_end.ptr, *of = (const int32_t *)t->b_p2p_off.ptr,
                  *sr = (const int32_t *)t->b_p2p_src.ptr, *mi = (const int32_t *)t->b_sym_mir.ptr;
    const uint32_t *rb = (const uint32_t *)t->b_sym_base.ptr;
    const float4 *o = (const float4 *)t->b_o32.ptr, *olo = o + t->n;
    float *rev = (float *)t->b_sym_rev.ptr;
    double *fwd = (double *)t->b_sym_fwd.ptr;
    auto run = [&](auto kern, auto gath) {
        kern<<<g, kSym32Threads, 0, st>>>(lv, bg, en, of, sr, mi, rb, (const int32_t *)t->b_level.ptr,
                                          (const int32_t *)t->b_cx.ptr, (const int32_t *)t->b_cy.ptr,
                                          (const int32_t *)t->b_cz.ptr, (const int32_t *)t->b_sys.ptr,
                                          (const double *)t->b_sysbox.ptr, o, olo, (const float *)t->b_S32.ptr,
                                          rev, fwd);
        gath<<<g, kSym32Threads, 0, st>>>(lv, bg, en, of, sr, mi, rb, rev, fwd, (const double *)t->b_phi.ptr,
                                          (const double *)t->b_E.ptr, (const int32_t *)t->b_perm.ptr, phi, E);
    };
    if (want_phi && want_field) run(k_p2p32_sym<S, true, true>, k_p2p32_sym_gather<true, true>);
    else if (want_phi) run(k_p2p32_sym<S, true, false>, k_p2p32_sym_gather<true, false>);
    else run(k_p2p32_sym<S, false, true>, k_p2p32_sym_gather<false, true>);
}

template <int S>
void launch_p2p32(fmm_tree *t, int want_phi, int want_field, double *phi, double *E)
{
    auto go = [&](auto kern) {
        kern<<<(unsigned)t->nleaves, kP2PThreads, 0, t->stream>>>(
            (const int32_t *)t->b_leaves.ptr, (const int32_t *)t->b_begin.ptr,
            (const int32_t *)t->b_end.ptr, (const int32_t *)t->b_p2p_off.ptr,
            (const int32_t *)t->b_p2p_src.ptr, (const int32_t *)t->b_level.ptr,
            (const int32_t *)t->b_cx.ptr, (const int32_t *)t->b_cy.ptr, (const int32_t *)t->b_cz.ptr,
            (const int32_t *)t->b_sys.ptr, (const double *)t->b_sysbox.ptr,
            (const double *)t->b_half.ptr,
            (const float4 *)t->b_o32.ptr, (const float4 *)t->b_o32.ptr + t->n,
            (const float *)t->b_S32.ptr, (const float *)t->b_S32.ptr + t->n * (t->nS == 6 ? 7 : t->nS),
            (const double *)t->b_phi.ptr, (const double *)t->b_E.ptr, (const int32_t *)t->b_perm.ptr,
            phi, E);
    };
    if (t->p2p_tt == 1) {
        if (want_phi && want_field) go(k_p2p32<S, true, true, 1>);
        else if (want_phi) go(k_p2p32<S, true, false, 1>);
        else go(k_p2p32<S, false, true, 1>);
    } else {
        if (want_phi && want_field) go(k_p2p32<S, true, true, 2>);
        else if (want_phi) go(k_p2p32<S, true, false, 2>);
        else go(k_p2p32<S, false, true, 2>);
    }
}

void record(fmm_tree *t, int i)
{
    if (t->profiling) cudaEventRecord(t->ev[i], t->stream);
}

fmm_status upload_consts32(fmm_tree *t)
{
    static int ready[64] = {0};
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (t->device < 64 && ready[t->device]) return FMM_OK;
    const MultiIndex &I = multi_index();
    int8_t x[kMaxTot], y[kMaxTot], z[kMaxTot];
    for (int i = 0; i < kMaxTot; ++i) { x[i] = (int8_t)I.nx[i]; y[i] = (int8_t)I.ny[i]; z[i] = (int8_t)I.nz[i]; }
    float inv[kMaxOrder + 2], invf[kMaxOrder + 1];
    inv[0] = 0.0f;
    for (int q = 1; q < kMaxOrder + 2; ++q) inv[q] = (float)(1.0 / q);
    double fct = 1.0;
    for (int q = 0; q <= kMaxOrder; ++q) { if (q) fct *= q; invf[q] = (float)(1.0 / fct); }
    FMM_TRY(cuda_check(t, cudaMemcpyToSymbol(x_nx, x, sizeof(x)), "constants"));
    FMM_TRY(cuda_check(t, cudaMemcpyToSymbol(x_ny, y, sizeof(y)), "constants"));
    FMM_TRY(cuda_check(t, cudaMemcpyToSymbol(x_nz, z, sizeof(z)), "constants"));
    FMM_TRY(cuda_check(t, cudaMemcpyToSymbol(x_invint, inv, sizeof(inv)), "constants"));
    FMM_TRY(cuda_check(t, cudaMemcpyToSymbol(x_invfact, invf, sizeof(invf)), "constants"));
    if (t->device < 64) ready[t->device] = 1;
    return FMM_OK;
}

}  // namespace

fmm_status run_mixed(fmm_tree *t, int p, int want_phi, int want_field, double *phi_out,
                     double *E_out)
{
    cudaStream_t st = t->stream;
    const int s = t->s;
    if (t->s_hi != t->s) {
        t->err = "mixed source orders are evaluated by the FP64 form";
        return FMM_EORDER;
    }
    FMM_TRY(upload_consts32(t));
    DevTables tb;
    const int32_t *lut;
    FMM_TRY(upload_tables(t, s, p, want_phi ? 0 : 1, &tb, &lut));
    const int64_t nc = t->ncells, n = t->n;
    const int P1 = p + 1;
    // cross-level M2L pairs scale FP32 values by 2^(gap * order): keep them in range
    if (t->max_gap * (p + s + 1) > 96) {
        t->err = "mixed precision: level gap " + std::to_string(t->max_gap) +
                 " of an M2L pair is too large for FP32 scaled expansions at this order";
        return FMM_EORDER;
    }
    FMM_TRY(build_dtables(t, p, tb, lut));
    // the buffers every evaluate of this form needs come first
    FMM_TRY(ensure(t, t->b_o32, 32 * (size_t)n));          // hi and lo float4 halves
    FMM_TRY(ensure(t, t->b_S32, 8 * (size_t)n * (t->nS == 6 ? 7 : t->nS)));   // hi, then lo
    FMM_TRY(ensure(t, t->b_M32, 4 * (size_t)nc * row4(tb.nM)));
    FMM_TRY(ensure(t, t->b_L32, 4 * (size_t)nc * tb.nLh));
    FMM_TRY(ensure(t, t->b_ud, 8 * (size_t)(nc + 1)));      // upward counters, downward flags
    FMM_TRY(ensure(t, t->b_phi, 8 * (size_t)n));
    FMM_TRY(ensure(t, t->b_E, 24 * (size_t)n));
    // The M2L this evaluate takes.  FMM_3XTF32: the tensor cores where the
    // operator fits them; otherwise (and in FMM_FP32) the SIMT FP32 M2L over the
    // same plan's tiles where its layout fits, else one block per target cell.
    // The plan and operator images must also fit the handle's memory budget
    // (decided when they are built, below).
    bool use_tc = t->n_m2l > 0 && t->prec == FMM_3XTF32 && !t->m2l_simt && tc_usable(t, s, p);
    const bool tile_ok = t->n_m2l > 0 && t->m2l_tiled && m32_usable(t, s, p, tb.harmonic, tb.n_lo);
    bool use_tile = false;
    auto prepare = [&]() -> fmm_status {
        if (use_tc) {
            const fmm_status pst = tc_prepare(t, p);
            if (pst == FMM_EBUDGET) {
                tc_release(t);
                t->err.clear();
                use_tc = false;
            } else {
                FMM_TRY(pst);
            }
        }
        use_tile = !use_tc && tile_ok;
        if (use_tile) {
            const fmm_status pst = m32_prepare(t, p);
            if (pst == FMM_EBUDGET) {
                tc_release(t);
                t->err.clear();
                use_tile = false;
            } else {
                FMM_TRY(pst);
            }
        }
        return FMM_OK;
    };
    // A plan that has to be built (new lists or p: its two host syncs) is
    // built on the handle's side stream while the upward pass runs; it needs
    // only the lists and the D table, both complete here.  Not while the
    // stream is being captured (the graph's evaluate follows an ordinary one,
    // which built the plan).
    const bool plan_stale = (use_tc && (!t->tc_plan || t->tc_img_p != p)) ||
                            (!use_tc && tile_ok && (!t->tc_plan || t->m32_img_p != p));
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (plan_stale) FMM_TRY(cuda_check(t, cudaStreamIsCapturing(st, &cap), "capture status"));
    const bool side = plan_stale && cap == cudaStreamCaptureStatusNone;
    if (side) {
        FMM_TRY(side_stream(t));
        FMM_TRY(cuda_check(t, cudaEventRecord(t->ev_lists, st), "event"));
    }
    record(t, 6);
    const int32_t *leaves = (const int32_t *)t->b_leaves.ptr;
    const int32_t *begin = (const int32_t *)t->b_begin.ptr, *end = (const int32_t *)t->b_end.ptr;
    const int32_t *cx = (const int32_t *)t->b_cx.ptr, *cy = (const int32_t *)t->b_cy.ptr,
                  *cz = (const int32_t *)t->b_cz.ptr;
    const double *half = (const double *)t->b_half.ptr;
    float4 *o = (float4 *)t->b_o32.ptr;
    float *S32 = (float *)t->b_S32.ptr, *M = (float *)t->b_M32.ptr, *L = (float *)t->b_L32.ptr;

    {
        // prep, P2M and M2M in one launch; the arrival counters start (and end) at zero
        cudaMemsetAsync(t->b_ud.ptr, 0, 4 * (size_t)nc, st);
        size_t smem = 4 * std::max<size_t>((size_t)kChunk * 3 * P1 + (size_t)kChunk * (tb.nK + 1) +
                                               (size_t)kChunk * 8 + 4,
                                           8 * ((size_t)tb.nK + tb.nM));
        allow_max_dynamic_smem(k_upward32);
        k_upward32<<<(unsigned)t->nleaves, 128, smem, st>>>(
            leaves, begin, end, (const int32_t *)t->b_parent.ptr, (const int32_t *)t->b_child.ptr,
            (const int32_t *)t->b_nchild.ptr, cx, cy, cz, half, (const double *)t->b_centre.ptr,
            (const double *)t->b_px.ptr, (const double *)t->b_py.ptr, (const double *)t->b_pz.ptr,
            (const double *)t->b_S.ptr, t->nS, n, o, S32, tb, M, (unsigned *)t->b_ud.ptr);
    }
    t->launches += 1;
    record(t, 7);
    cudaMemsetAsync(L, 0, 4 * (size_t)nc * tb.nLh, st);
    // harmonic M2L: the folded multipoles, for either M2L
    const float *Ms = M;
    if (t->n_m2l > 0 && tb.harmonic) {
        FMM_TRY(ensure(t, t->b_Mh32, 4 * (size_t)nc * row4(tb.nMh)));
        launch_fold_m(st, M, row4(tb.nM), nc, tb, (float *)t->b_Mh32.ptr, row4(tb.nMh));
        ++t->launches;
        Ms = (const float *)t->b_Mh32.ptr;
    }
    record(t, 8);
    if (side) {
        cudaStreamWaitEvent(t->side_st, t->ev_lists, 0);
        t->stream = t->side_st;
        const fmm_status ps = prepare();
        t->stream = st;
        cudaEventRecord(t->ev_plan, t->side_st);
        cudaStreamWaitEvent(st, t->ev_plan, 0);
        FMM_TRY(ps);
    } else {
        FMM_TRY(prepare());
    }
    if (t->n_m2l > 0 && !use_tc && !use_tile && t->d32_p != p && t->n_doff > 0) {
        FMM_TRY(ensure(t, t->b_D32, 4 * (size_t)t->n_doff * row4(tb.nD)));
        k_dtables32<<<gridm(t->n_doff * tb.nD, 256), 256, 0, st>>>(
            (const uint64_t *)t->b_dkeys.ptr, t->n_doff, tb.nD, (const double *)t->b_D.ptr, tb.mi,
            (float *)t->b_D32.ptr);
        ++t->launches;
        t->d32_p = p;
    }
    if (t->n_m2l > 0 && use_tc) {
        FMM_TRY(run_m2l_tc(t, p, Ms, row4(tb.nMh), tb.nMh, tb.nL, tb, L));
    } else if (t->n_m2l > 0 && use_tile) {
        FMM_TRY(run_m2l32_tile(t, p, Ms, row4(tb.nMh), tb, L));
    } else if (t->n_m2l > 0) {
        const int ldM = tb.nMh | 1, ldD = tb.nD | 1;
        size_t smem = 8 * (size_t)tb.m2l_slots * kM2LThreads +
                      4 * ((size_t)kBatch * (ldM + ldD) + (size_t)tb.m2l_T * kM2LThreads);
        allow_max_dynamic_smem(k_m2l32);
        k_m2l32<<<(unsigned)nc, kM2LThreads, smem, st>>>(
            (const int32_t *)t->b_m2l_off.ptr, (const int32_t *)t->b_m2l_src.ptr,
            (const int32_t *)t->b_m2l_didx.ptr, (const int32_t *)t->b_level.ptr, Ms,
            (const float *)t->b_D32.ptr, tb, L);
        ++t->launches;
    }
    record(t, 9);
    // L2L downward, all levels in one launch (flags and claim counter start at
    // zero), each leaf's L2P in the block that finishes its expansion; a
    // one-level tree has no shifts and takes the L2P on its own
    if (t->nlevels > 1) {
        unsigned *ctl = (unsigned *)t->b_ud.ptr + nc + 1;
        cudaMemsetAsync(ctl, 0, 4 * (size_t)(nc + 1), st);
        const int64_t nint = nc - t->nleaves;        // cells with children: after the leaves in b_leaves
        const int32_t *parent = (const int32_t *)t->b_parent.ptr;
        if (nint > 0) {
            const size_t smem_i = 4 * ((size_t)tb.nK + tb.nL);
            allow_max_dynamic_smem(k_downward32);
            k_downward32<<<(unsigned)nint, 128, smem_i, st>>>(nint, leaves + t->nleaves, parent, cx, cy, cz,
                                                               tb, L, ctl);
            ++t->launches;
        }
        const size_t smem = 4 * std::max<size_t>((size_t)tb.nK + tb.nL, (size_t)tb.nL + kL2PThreads * 3 * P1);
        allow_max_dynamic_smem(k_downward32_leaf);
        k_downward32_leaf<<<(unsigned)t->nleaves, 128, smem, st>>>(
            leaves, parent, cx, cy, cz, tb, L, begin, end, half, o, want_phi, want_field, (double *)t->b_phi.ptr,
            (double *)t->b_E.ptr);
        ++t->launches;
        record(t, 10);
    } else {
        record(t, 10);
        const size_t smem = 4 * (size_t)(tb.nL + kL2PThreads * 3 * P1);
        allow_max_dynamic_smem(k_l2p32);
        k_l2p32<<<(unsigned)t->nleaves, kL2PThreads, smem, st>>>(
            leaves, begin, end, half, o, L, tb, want_phi, want_field, (double *)t->b_phi.ptr,
            (double *)t->b_E.ptr);
        ++t->launches;
    }
    record(t, 11);
    if (t->p2p_variant == 2) {             // symmetric near field (the reverse rows hold floats)
        const fmm_status ps = sym_prepare(t, (want_phi ? 1 : 0) + (want_field ? 3 : 0));
        if (ps == FMM_OK && t->sym_rows >= 0) {
            switch (s) {
            case 0: launch_p2p32_sym<0>(t, want_phi, want_field, phi_out, E_out); break;
            case 1: launch_p2p32_sym<1>(t, want_phi, want_field, phi_out, E_out); break;
            default: launch_p2p32_sym<2>(t, want_phi, want_field, phi_out, E_out); break;
            }
            t->launches += 2;
            return cuda_check(t, cudaGetLastError(), "mixed-precision kernels");
        }
        if (ps != FMM_OK && ps != FMM_EBUDGET) return ps;
        t->err.clear();                       // over the budget: the one-way kernel
    }
    switch (s) {
    case 0: launch_p2p32<0>(t, want_phi, want_field, phi_out, E_out); break;
    case 1: launch_p2p32<1>(t, want_phi, want_field, phi_out, E_out); break;
    default: launch_p2p32<2>(t, want_phi, want_field, phi_out, E_out); break;
    }
    ++t->launches;
    return cuda_check(t, cudaGetLastError(), "mixed-precision kernels");
}

}  // namespace fmm
