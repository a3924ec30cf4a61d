// operators.cu -- derivative tables and the expansion operators (FP64).
//
// Conventions (paper §2, read as stated in the header):
//   P2M  M_m(z)   = sum_j sum_{|a|=s, a<=m} (z - x_j)^(m-a)/(m-a)! S_{j,a}   (Eq. (5))
//   M2M  M_n(z')  = sum_{k<=n} (z' - z)^k/k! M_{n-k}(z)                        (Eq. (4))
//   M2L  L_n(zt)  = sum_{m, |n|+|m|<=p+s} D_{n+m}(zt - zs) M_m(zs)            (Eq. (8))
//   L2L  L_n(z')  = sum_{|n+k|<=p} (z' - z)^k/k! L_{n+k}(z)
//   L2P  phi = sum_n (x-z)^n/n! L_n,  d_k phi = sum_{n>=e_k} (x-z)^(n-e_k)/(n-e_k)! L_n
//                                                                             (Eqs. (9), (10))
// D_n(R) = grad^n (1/|R|) is generated once per distinct M2L offset.
#include <algorithm>
#include <cstring>
#include <stdexcept>
#include <mutex>

#include "fmm_internal.cuh"

namespace fmm {

MultiIndex::MultiIndex()
{
    std::memset(lut, 0xff, sizeof(lut));
    int i = 0;
    for (int k = 0; k <= kMaxOrder; ++k)
        for (int a = 0; a <= k; ++a)          // a = ny + nz
            for (int z = 0; z <= a; ++z) {
                nx[i] = k - a; ny[i] = a - z; nz[i] = z;
                lut[k - a][a - z][z] = (int16_t)i;
                ++i;
            }
}

const MultiIndex &multi_index()
{
    static MultiIndex mi;
    return mi;
}

void build_tables(OpTables &T, int s, int s_hi, int p, int n_lo, int m2l_threads, bool harmonic)
{
    const MultiIndex &I = multi_index();
    T.s = s; T.p = p; T.n_lo = n_lo; T.harmonic = harmonic;
    // source terms a: the orders s..s_hi, graded indices from ntot(s - 1) on
    T.nS = ntot(s_hi) - ntot(s - 1); T.m0 = ntot(s - 1); T.nM = ntot(p + s) - T.m0; T.nL = ntot(p);
    T.nD = ntot(p + s);
    const int nK = ntot(p);                   // shift / particle monomials |k| <= p

    T.p2m_terms.assign((size_t)T.nM * T.nS, -1);
    for (int mi = 0; mi < T.nM; ++mi) {
        const int m = mi + T.m0;
        for (int ai = 0; ai < T.nS; ++ai) {
            const int a = ai + T.m0;
            int kx = I.nx[m] - I.nx[a], ky = I.ny[m] - I.ny[a], kz = I.nz[m] - I.nz[a];
            if (kx >= 0 && ky >= 0 && kz >= 0) T.p2m_terms[(size_t)mi * T.nS + ai] = I(kx, ky, kz);
        }
    }
    T.mono_par.assign(nK, 0); T.mono_axis.assign(nK, 0); T.mono_pow.assign(nK, 0);

    T.m2m_off.assign(1, 0); T.m2m_k.clear(); T.m2m_q.clear();
    for (int ni = 0; ni < T.nM; ++ni) {
        const int n = ni + T.m0;
        for (int qi = 0; qi < T.nM; ++qi) {
            const int q = qi + T.m0;
            int kx = I.nx[n] - I.nx[q], ky = I.ny[n] - I.ny[q], kz = I.nz[n] - I.nz[q];
            if (kx < 0 || ky < 0 || kz < 0) continue;
            T.m2m_k.push_back(I(kx, ky, kz));
            T.m2m_q.push_back(qi);
        }
        T.m2m_off.push_back((int)T.m2m_k.size());
    }
    T.l2l_off.assign(1, 0); T.l2l_k.clear(); T.l2l_q.clear();
    for (int n = 0; n < T.nL; ++n) {
        for (int k = 0; k < nK; ++k) {
            int qx = I.nx[n] + I.nx[k], qy = I.ny[n] + I.ny[k], qz = I.nz[n] + I.nz[k];
            if (qx + qy + qz > p) continue;
            T.l2l_k.push_back(k);
            T.l2l_q.push_back(I(qx, qy, qz));
        }
        T.l2l_off.push_back((int)T.l2l_k.size());
    }
    const int nG = ntot(p - 1);
    T.l2p_grad.assign((size_t)3 * std::max(nG, 0), 0);
    for (int k = 0; k < nG; ++k) {
        T.l2p_grad[3 * k + 0] = I(I.nx[k] + 1, I.ny[k], I.nz[k]);
        T.l2p_grad[3 * k + 1] = I(I.nx[k], I.ny[k] + 1, I.nz[k]);
        T.l2p_grad[3 * k + 2] = I(I.nx[k], I.ny[k], I.nz[k] + 1);
    }

    // ---- harmonic M2L (§3.1 harmonic derivatives).  Since D_{k+2x} + D_{k+2y}
    // + D_{k+2z} = 0 for every k, a term D_{n+m} M_m with m_z >= 2 equals
    // -(D_{n+m-2z+2x} + D_{n+m-2z+2y}) M_m, a pair of terms of the same degree
    // |m|, hence inside the same truncation |n| + |m| <= p + s: moving M_m onto
    // those two m (in decreasing m_z) leaves the m with m_z <= 1 only, 2k+1
    // per degree k.  Likewise L_n with n_z >= 2 is -L_{n+2x-2z} - L_{n+2y-2z}
    // (same degree, same m range).  The same sums, mathematically.
    T.h_rm.clear();
    for (int mi = 0; mi < T.nM; ++mi)
        if (!harmonic || I.nz[mi + T.m0] <= 1) T.h_rm.push_back(mi);
    T.nMh = (int)T.h_rm.size();
    std::vector<int> r_of(T.nM, -1);
    for (int r = 0; r < T.nMh; ++r) r_of[T.h_rm[r]] = r;
    T.h_fold.clear(); T.h_fold_off.assign(1, 0);
    T.h_unfold.clear(); T.h_unfold_off.assign(1, 0);
    if (harmonic) {
        for (int z = p + s - 2; z >= 0; --z) {
            for (int mi = 0; mi < T.nM; ++mi) {
                const int m = mi + T.m0;
                if (I.nz[m] != z) continue;
                const int a = I.nx[m] >= 2 ? I(I.nx[m] - 2, I.ny[m], I.nz[m] + 2) - T.m0 : -1;
                const int b = I.ny[m] >= 2 ? I(I.nx[m], I.ny[m] - 2, I.nz[m] + 2) - T.m0 : -1;
                if (a < 0 && b < 0) continue;
                T.h_fold.insert(T.h_fold.end(), {mi, a, b});
            }
            T.h_fold_off.push_back((int)T.h_fold.size() / 3);
        }
        for (int z = 2; z <= p; ++z) {
            for (int n = 0; n < T.nL; ++n) {
                if (I.nz[n] != z) continue;
                T.h_unfold.insert(T.h_unfold.end(), {n, I(I.nx[n] + 2, I.ny[n], z - 2),
                                                     I(I.nx[n], I.ny[n] + 2, z - 2)});
            }
            T.h_unfold_off.push_back((int)T.h_unfold.size() / 3);
        }
    }
    // stored locals: the n with n_z <= 1 when harmonic (the others follow from
    // the identity wherever the full expansion is needed), all of them otherwise
    T.h_rn.clear();
    for (int n = 0; n < T.nL; ++n)
        if (!harmonic || I.nz[n] <= 1) T.h_rn.push_back(n);
    T.nLh = (int)T.h_rn.size();

    // ---- M2L: flat (n, m) term list in n order, cut into equal per-thread
    // chunks; each maximal same-n run inside a chunk owns one partial slot.
    // m is the position r in the kept list h_rm (all m when not harmonic).
    struct Term { int n, m, d; };
    std::vector<Term> terms;
    for (int n = 0; n < T.nL; ++n) {
        const int kn = I.nx[n] + I.ny[n] + I.nz[n];
        if (kn < n_lo || (harmonic && I.nz[n] > 1)) continue;
        for (int r = 0; r < T.nMh; ++r) {
            const int m = T.h_rm[r] + T.m0;
            if (kn + I.nx[m] + I.ny[m] + I.nz[m] > p + s) continue;
            terms.push_back({n, r, I(I.nx[n] + I.nx[m], I.ny[n] + I.ny[m], I.nz[n] + I.nz[m])});
        }
    }
    const int W = (int)terms.size(), Tn = m2l_threads;
    const int cap = std::max(1, (W + Tn - 1) / Tn);
    T.m2l_threads = Tn; T.m2l_T = cap;
    T.m2l_desc.assign((size_t)cap * Tn, 0xffffffffu);
    std::vector<std::vector<int>> red(T.nL);
    int max_slots = 0;
    for (int j = 0; j < Tn; ++j) {
        const int b = j * cap, e = std::min(W, b + cap);
        int slot = -1;
        for (int i = b; i < e; ++i) {
            if (i == b || terms[i].n != terms[i - 1].n) {
                ++slot;
                red[terms[i].n].push_back(slot * Tn + j);
            }
            const bool flush = (i + 1 == e) || terms[i + 1].n != terms[i].n;
            T.m2l_desc[(size_t)(i - b) * Tn + j] =
                (uint32_t)terms[i].m | ((uint32_t)terms[i].d << 9) | ((uint32_t)flush << 18) |
                ((uint32_t)slot << 19);
        }
        max_slots = std::max(max_slots, slot + 1);
    }
    T.m2l_slots = max_slots;
    T.m2l_red_off.assign(1, 0); T.m2l_red_src.clear();
    for (int n = 0; n < T.nL; ++n) {
        for (int v : red[n]) T.m2l_red_src.push_back(v);
        T.m2l_red_off.push_back((int)T.m2l_red_src.size());
    }
}

namespace {

constexpr int kM2LThreads = 128;
constexpr int kM2LBatch = 16;

__constant__ int8_t c_nx[kMaxTot], c_ny[kMaxTot], c_nz[kMaxTot];


// ---------------------------------------------------- derivative tables
// r^2 D_n = -(2 n_i - 1) R_i D_{n-e_i} - (n_i - 1)^2 D_{n-2e_i}
//           - sum_{j != i} [ 2 n_j R_j D_{n-e_j} + n_j (n_j - 1) D_{n-2e_j} ],
// i = first axis with n_i >= 1 (Leibniz' rule on r^2 d_i(1/r) = -R_i / r).
// Rows are unit-free: D_k(v) at the integer offset v of the key; a pair with
// finer half-cell u uses u^-(|k|+1) D_k(v), applied exactly as an exponent shift.
// One warp per distinct offset: the row is built shell by shell in the warp's
// shared memory (an entry of shell |n| reads shells |n| - 1 and |n| - 2 only,
// so a shell's entries are independent and the lanes take them side by side),
// then stored.  Each entry is the same arithmetic as a one-thread recurrence.
__global__ void k_dtables(const uint64_t *dkeys, int64_t ndoff, int nD, const int32_t *lut,
                          double *D)
{
    extern __shared__ double dsm[];
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= ndoff) return;
    double *Dr = dsm + (threadIdx.x >> 5) * (int64_t)nD;
    const uint64_t key = dkeys[r];
    double R[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        R[i] = (double)((long long)((key >> (34 - 17 * i)) & 0x1ffffull) - kKeyBias);
    const double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    const double inv_r2 = 1.0 / r2;
    if (lane == 0) Dr[0] = rsqrt(r2);
    __syncwarp();
    const int L = kMaxOrder + 1;
    for (int sh = 1, s0 = 1; s0 < nD; ++sh) {
        const int s1 = min(nD, (sh + 1) * (sh + 2) * (sh + 3) / 6);      // shell sh: [s0, s1)
        for (int idx = s0 + lane; idx < s1; idx += 32) {
            const int n[3] = {c_nx[idx], c_ny[idx], c_nz[idx]};
            const int i = n[0] ? 0 : (n[1] ? 1 : 2);
            int m[3] = {n[0], n[1], n[2]};
            m[i] -= 1;
            double acc = -(2.0 * n[i] - 1.0) * R[i] * Dr[lut[(m[0] * L + m[1]) * L + m[2]]];
            if (n[i] >= 2) {
                int q[3] = {m[0], m[1], m[2]};
                q[i] -= 1;
                acc -= (double)((n[i] - 1) * (n[i] - 1)) * Dr[lut[(q[0] * L + q[1]) * L + q[2]]];
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (j == i || n[j] == 0) continue;
                int q[3] = {n[0], n[1], n[2]};
                q[j] -= 1;
                acc -= 2.0 * n[j] * R[j] * Dr[lut[(q[0] * L + q[1]) * L + q[2]]];
                if (n[j] >= 2) {
                    q[j] -= 1;
                    acc -= (double)(n[j] * (n[j] - 1)) * Dr[lut[(q[0] * L + q[1]) * L + q[2]]];
                }
            }
            Dr[idx] = acc * inv_r2;
        }
        __syncwarp();
        s0 = s1;
    }
    for (int k = lane; k < nD; k += 32) D[r * nD + k] = Dr[k];
}

// per-axis scaled powers d^j / j!, j <= P, then monomials d^k / k! = ax[kx] ay[ky] az[kz]
__constant__ double c_invint[kMaxOrder + 2];     // 1/j

__device__ __forceinline__ void axis_powers(double d, int P, double *out)
{
    double v = 1.0;
    out[0] = 1.0;
    for (int j = 1; j <= P; ++j) {
        v = v * d * c_invint[j];
        out[j] = v;
    }
}

// ------------------------------------------------------------------ P2M
constexpr int kP2MThreads = 128;
constexpr int kP2MChunk = 16;
constexpr int kP2MPer = 4;                // up to 4 * 128 = 512 M components
// source terms of one particle: the kernel is instantiated for 3, 6 and 10 (one
// order up to a dipole, a quadrupole, mixed orders) and takes the smallest that fits

// One block per leaf.  Each thread owns up to kP2MPer components m and keeps
// the monomial index of m - a for each source term a in registers (an absent
// term points at a zero slot), so the particle loop is branch-free.
template <int kMaxSrc>
__device__ __forceinline__ void p2m_leaf(int c, const int32_t *begin, const int32_t *end,
                                         const double *centre, const double *px, const double *py,
                                         const double *pz, const double *S, const DevTables &tb,
                                         double *M, double *sm)
{
    const int P = tb.p, P1 = tb.p + 1, nK = tb.nK, nK1 = tb.nK + 1, nS = tb.nS;
    double *apow = sm;                                  // [chunk][3][P+1]
    double *mono = apow + kP2MChunk * 3 * P1;           // [chunk][nK + 1], last = 0
    double *Ssm = mono + kP2MChunk * nK1;               // [chunk][nS]
    const int b = begin[c], e = end[c];
    const double z0 = centre[3 * c], z1 = centre[3 * c + 1], z2 = centre[3 * c + 2];
    int kt[kP2MPer][kMaxSrc];
    double acc[kP2MPer];
#pragma unroll
    for (int u = 0; u < kP2MPer; ++u) {
        acc[u] = 0.0;
        const int mi = threadIdx.x + u * kP2MThreads;
#pragma unroll
        for (int a = 0; a < kMaxSrc; ++a) {
            const int k = (mi < tb.nM && a < nS) ? tb.p2m_terms[mi * nS + a] : -1;
            kt[u][a] = k >= 0 ? k : nK;
        }
    }
    for (int j0 = b; j0 < e; j0 += kP2MChunk) {
        const int nj = min(kP2MChunk, e - j0);
        for (int t = threadIdx.x; t < 3 * nj; t += blockDim.x) {
            const int j = t / 3, ax = t % 3;
            const double x = ax == 0 ? px[j0 + j] : (ax == 1 ? py[j0 + j] : pz[j0 + j]);
            const double zc = ax == 0 ? z0 : (ax == 1 ? z1 : z2);
            axis_powers(zc - x, P, apow + (j * 3 + ax) * P1);
        }
        for (int t = threadIdx.x; t < nj * nS; t += blockDim.x)
            Ssm[t] = S[(int64_t)j0 * nS + t];
        __syncthreads();
        // each thread its monomials k (exponents decoded once) for every particle
        for (int k = threadIdx.x; k < nK1; k += blockDim.x) {
            int ox = 0, oy = 0, oz = 0;
            if (k < nK) {
                const int v = mi_at(tb.mi, k);
                ox = mi_nx(v); oy = P1 + mi_ny(v); oz = 2 * P1 + mi_nz(v);
            }
            for (int j = 0; j < nj; ++j) {
                const double *a = apow + j * 3 * P1;
                mono[j * nK1 + k] = k < nK ? a[ox] * a[oy] * a[oz] : 0.0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kP2MPer; ++u) {
            if (threadIdx.x + u * kP2MThreads >= tb.nM) break;
            for (int j = 0; j < nj; ++j) {
                const double *mj = mono + j * nK1, *sj = Ssm + j * nS;
#pragma unroll
                for (int a = 0; a < kMaxSrc; ++a)
                    if (a < nS) acc[u] = fma(mj[kt[u][a]], sj[a], acc[u]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < kP2MPer; ++u) {
        const int mi = threadIdx.x + u * kP2MThreads;
        if (mi < tb.nM) M[(int64_t)c * tb.nM + mi] = acc[u];
    }
}

// ------------------------------------------------------------------ M2M
// The multipole of parent cell c from its children (Eq. (4) with the sign of
// R2), children summed in index order.  ldcg: the children's rows may have been
// written by other blocks of the same launch.
__device__ __forceinline__ void m2m_cell(int c, const int32_t *child, const int32_t *nchild,
                                         const double *centre, const DevTables &tb, double *M,
                                         double *sm)
{
    const int P = tb.p, nK = tb.nK;
    double *apow = sm;                  // [3][P+1]
    double *mono = apow + 3 * (P + 1);  // [nK]
    double *Mc = mono + nK;             // [nM]
    const int nch = nchild[c];
    double acc[kP2MPer];
#pragma unroll
    for (int u = 0; u < kP2MPer; ++u) acc[u] = 0.0;
    for (int i = 0; i < nch; ++i) {
        const int ch = child[c] + i;
        if (threadIdx.x < 3)
            axis_powers(centre[3 * c + threadIdx.x] - centre[3 * ch + threadIdx.x], P,
                        apow + threadIdx.x * (P + 1));
        for (int t = threadIdx.x; t < tb.nM; t += blockDim.x) Mc[t] = __ldcg(M + (int64_t)ch * tb.nM + t);
        __syncthreads();
        for (int k = threadIdx.x; k < nK; k += blockDim.x) {
            const int v = mi_at(tb.mi, k);
            mono[k] = apow[mi_nx(v)] * apow[(P + 1) + mi_ny(v)] * apow[2 * (P + 1) + mi_nz(v)];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kP2MPer; ++u) {
            const int ni = threadIdx.x + u * 128;
            if (ni >= tb.nM) break;
            for (int q = tb.m2m_off[ni]; q < tb.m2m_off[ni + 1]; ++q)
                acc[u] = fma(mono[tb.m2m_k[q]], Mc[tb.m2m_q[q]], acc[u]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < kP2MPer; ++u) {
        const int ni = threadIdx.x + u * 128;
        if (ni < tb.nM) M[(int64_t)c * tb.nM + ni] = acc[u];
    }
}

// The upward pass in one launch: block b forms the multipole of leaf b (P2M,
// Eq. (3)), then climbs -- the block whose child arrives last at a parent
// (a counter per cell) forms that parent's multipole (M2M), and so on up to
// the root.  No block waits on another; every parent is formed exactly once,
// from its finished children, in the same order as a level-by-level pass.
// arrive[] starts at zero and is left at zero (the winner resets it).
template <int kMaxSrc>
__global__ void __launch_bounds__(kP2MThreads)
k_upward(const int32_t *leaves, const int32_t *begin, const int32_t *end, const int32_t *parent,
         const int32_t *child, const int32_t *nchild, const double *centre, const double *px,
         const double *py, const double *pz, const double *S, DevTables tb, double *M,
         unsigned *arrive)
{
    extern __shared__ double sm[];
    __shared__ int s_go;
    int c = leaves[blockIdx.x];
    p2m_leaf<kMaxSrc>(c, begin, end, centre, px, py, pz, S, tb, M, sm);
    for (;;) {
        const int pa = parent[c];
        if (pa < 0) break;
        __syncthreads();                       // every thread's row of c is written
        if (threadIdx.x == 0) {
            __threadfence();                   // ... and visible before the arrival counts
            const unsigned n = atomicAdd(&arrive[pa], 1u) + 1u;
            const bool last = n == (unsigned)nchild[pa];
            if (last) {
                arrive[pa] = 0u;
                __threadfence();               // the other children's rows are visible now
            }
            s_go = last;
        }
        __syncthreads();
        if (!s_go) break;
        m2m_cell(pa, child, nchild, centre, tb, M, sm);
        c = pa;
    }
}

// ------------------------------------------------------------------ M2L
// One block per target cell.  Sources are taken kM2LBatch at a time: their
// multipoles and derivative-table rows are staged in shared memory, then
// each thread walks its fixed chunk of (n, m) terms, accumulating
// D_{n+m} M_m over the staged sources, and flushes each finished n-run to its
// partial slot.  Partials are summed per n in a fixed order at the end.
// x * 2^e for normal x (exponent field arithmetic; zeros stay zero)
__device__ __forceinline__ double scale_pow2(double x, int e)
{
    const long long b = __double_as_longlong(x);
    return (b & 0x7ff0000000000000ll) ? __longlong_as_double(b + ((long long)e << 52)) : x;
}

// One warp per cell: the row of M in shared memory (FP64), the fold levels of
// the harmonic M2L in order (an entry reads only entries of the level two
// z-steps up, final by then), the kept entries written in graded order.
template <typename Tm>
__global__ void __launch_bounds__(128)
k_fold_m(const Tm *M, int ldM, int64_t nc, DevTables tb, Tm *Mh, int ldH)
{
    extern __shared__ double fsm[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = blockIdx.x * 4ll + w;
    if (c >= nc) return;                 // whole warps; no block barrier below
    double *v = fsm + w * tb.nM;
    for (int m = lane; m < tb.nM; m += 32) v[m] = (double)M[c * ldM + m];
    __syncwarp();
    for (int l = 0; l < tb.h_fold_lev; ++l) {
        for (int q = tb.h_fold_off[l] + lane; q < tb.h_fold_off[l + 1]; q += 32) {
            const int i = tb.h_fold[3 * q], a = tb.h_fold[3 * q + 1], b = tb.h_fold[3 * q + 2];
            double x = v[i];
            if (a >= 0) x -= v[a];
            if (b >= 0) x -= v[b];
            v[i] = x;
        }
        __syncwarp();
    }
    for (int r = lane; r < tb.nMh; r += 32) Mh[c * ldH + r] = (Tm)v[tb.h_rm[r]];
}

__global__ void __launch_bounds__(kM2LThreads)
k_m2l(const int32_t *off, const int32_t *src, const int32_t *didx, const int32_t *level,
      const int32_t *sys, const int *e_side, const double *M, const double *D, DevTables tb,
      double *L)
{
    extern __shared__ double sm[];
    const int c = blockIdx.x;
    const int b = off[c], e = off[c + 1];
    if (b == e) return;
    // M: the kept (folded, when harmonic) multipole rows, nMh per cell
    const int nM = tb.nMh, nD = tb.nD, T = tb.m2l_T, Tn = kM2LThreads;
    const int ldM = nM | 1, ldD = nD | 1;              // odd strides spread banks
    double *Msm = sm;                                  // [batch][ldM]
    double *Dsm = Msm + kM2LBatch * ldM;               // [batch][ldD]
    double *part = Dsm + kM2LBatch * ldD;              // [slots][Tn]
    uint32_t *desc = (uint32_t *)(part + tb.m2l_slots * Tn);   // [T][Tn]
    const int tid = threadIdx.x;
    const int lt = level[c], es = e_side[sys[c]];
    __shared__ int bsrc[kM2LBatch], bdidx[kM2LBatch], beu[kM2LBatch];
    for (int i = tid; i < T * Tn; i += Tn) desc[i] = tb.m2l_desc[i];
    for (int i = tid; i < tb.m2l_slots * Tn; i += Tn) part[i] = 0.0;
    for (int k0 = b; k0 < e; k0 += kM2LBatch) {
        const int kb = min(kM2LBatch, e - k0);
        __syncthreads();
        if (tid < kb) {                    // batch metadata, loaded in parallel
            const int s = src[k0 + tid];
            bsrc[tid] = s;
            bdidx[tid] = didx[k0 + tid];
            // u = side / 2^(lf+1): D_k(u v) = 2^(-(|k|+1) log2 u) D_k(v)
            beu[tid] = es - max(lt, level[s]) - 1;
        }
        __syncthreads();
        for (int k = 0; k < kb; ++k) {
            const double *Ms = M + (int64_t)bsrc[k] * nM;
            for (int m = tid; m < nM; m += Tn) Msm[k * ldM + m] = Ms[m];
            const double *Dk = D + (int64_t)bdidx[k] * nD;
            const int eu = beu[k];
            for (int d = tid; d < nD; d += Tn)
                Dsm[k * ldD + d] = scale_pow2(Dk[d], -(mi_shell(mi_at(tb.mi, d)) + 1) * eu);
        }
        __syncthreads();
        double acc = 0.0;
        for (int t = 0; t < T; ++t) {
            const uint32_t u = desc[t * Tn + tid];
            if (u == 0xffffffffu) break;
            const double *Mp = Msm + (u & 511u);
            const double *Dp = Dsm + ((u >> 9) & 511u);
            int k = 0;
            for (; k + 4 <= kb; k += 4) {
                acc = fma(Dp[k * ldD], Mp[k * ldM], acc);
                acc = fma(Dp[(k + 1) * ldD], Mp[(k + 1) * ldM], acc);
                acc = fma(Dp[(k + 2) * ldD], Mp[(k + 2) * ldM], acc);
                acc = fma(Dp[(k + 3) * ldD], Mp[(k + 3) * ldM], acc);
            }
            for (; k < kb; ++k) acc = fma(Dp[k * ldD], Mp[k * ldM], acc);
            if (u & (1u << 18)) {
                part[(u >> 19) * Tn + tid] += acc;
                acc = 0.0;
            }
        }
    }
    __syncthreads();
    // the stored components (n_z <= 1 when harmonic, the traceless form)
    for (int r = tid; r < tb.nLh; r += Tn) {
        const int n = tb.h_rn[r];
        double v = 0.0;
        for (int q = tb.m2l_red_off[n]; q < tb.m2l_red_off[n + 1]; ++q) v += part[tb.m2l_red_src[q]];
        L[(int64_t)c * tb.nLh + r] = v;
    }
}

// ------------------------------------------------------------------ L2L
// The local expansion of cell c shifted from its parent's (Eq. (9)-type Taylor
// shift), added to c's stored components.
__device__ __forceinline__ void l2l_cell(int c, int pa, const double *centre, const DevTables &tb,
                                         double *L, double *sm)
{
    const int P = tb.p, nK = tb.nK;
    double *apow = sm;
    double *mono = apow + 3 * (P + 1);
    double *Lp = mono + nK;
    if (threadIdx.x < 3)
        axis_powers(centre[3 * c + threadIdx.x] - centre[3 * pa + threadIdx.x], P,
                    apow + threadIdx.x * (P + 1));
    expand_local_cg(L + (int64_t)pa * tb.nLh, tb, Lp);        // the parent's full expansion
    for (int k = threadIdx.x; k < nK; k += blockDim.x) {
        const int v = mi_at(tb.mi, k);
        mono[k] = apow[mi_nx(v)] * apow[(P + 1) + mi_ny(v)] * apow[2 * (P + 1) + mi_nz(v)];
    }
    __syncthreads();
    // the child's stored components (the shift keeps the expansion harmonic)
    for (int r = threadIdx.x; r < tb.nLh; r += blockDim.x) {
        const int n = tb.h_rn[r];
        const int kn = mi_shell(mi_at(tb.mi, n));
        if (kn < tb.n_lo) continue;
        double acc = 0.0;
        for (int q = tb.l2l_off[n]; q < tb.l2l_off[n + 1]; ++q)
            acc = fma(mono[tb.l2l_k[q]], Lp[tb.l2l_q[q]], acc);
        L[(int64_t)c * tb.nLh + r] += acc;
    }
}

// ------------------------------------------------------------------ L2P
constexpr int kL2PThreads = 128;

// Leaf c: the far-field part of phi and E = -grad phi at its particles (Eqs.
// (9), (10)), one thread per particle, in sorted particle order.
__device__ __forceinline__ void l2p_leaf(int c, const int32_t *begin, const int32_t *end,
                                         const double *centre, const double *px, const double *py,
                                         const double *pz, const double *L, const DevTables &tb,
                                         int want_phi, int want_field, double *phi, double *E,
                                         double *sm)
{
    const int P = tb.p, P1 = tb.p + 1;
    double *Lsm = sm;                                       // [nL]
    double *a = Lsm + tb.nL + threadIdx.x * 3 * P1;         // this thread's [3][P+1]
    const int b = begin[c], e = end[c];
    expand_local_cg(L + (int64_t)c * tb.nLh, tb, Lsm);
    const double z0 = centre[3 * c], z1 = centre[3 * c + 1], z2 = centre[3 * c + 2];
    for (int j = b + threadIdx.x; j < e; j += blockDim.x) {
        axis_powers(px[j] - z0, P, a);
        axis_powers(py[j] - z1, P, a + P1);
        axis_powers(pz[j] - z2, P, a + 2 * P1);
        if (want_phi) {
            double f = 0.0;
            for (int k = 0; k < tb.nL; ++k)
                f = fma(a[c_nx[k]] * a[P1 + c_ny[k]] * a[2 * P1 + c_nz[k]], Lsm[k], f);
            phi[j] = f;
        }
        if (want_field) {
            double g0 = 0.0, g1 = 0.0, g2 = 0.0;
            for (int k = 0; k < tb.nG; ++k) {
                const double m = a[c_nx[k]] * a[P1 + c_ny[k]] * a[2 * P1 + c_nz[k]];
                g0 = fma(m, Lsm[tb.l2p_grad[3 * k]], g0);
                g1 = fma(m, Lsm[tb.l2p_grad[3 * k + 1]], g1);
                g2 = fma(m, Lsm[tb.l2p_grad[3 * k + 2]], g2);
            }
            E[3 * (int64_t)j] = -g0;
            E[3 * (int64_t)j + 1] = -g1;
            E[3 * (int64_t)j + 2] = -g2;
        }
    }
}


__global__ void __launch_bounds__(kL2PThreads)
k_l2p(const int32_t *leaves, const int32_t *begin, const int32_t *end, const double *centre,
      const double *px, const double *py, const double *pz, const double *L, DevTables tb,
      int want_phi, int want_field, double *phi, double *E)
{
    extern __shared__ double sm[];
    l2p_leaf(leaves[blockIdx.x], begin, end, centre, px, py, pz, L, tb, want_phi, want_field, phi, E, sm);
}

// The L2L shifts of all levels in one launch.  Blocks claim cells in
// breadth-first order (a counter), so a cell's parent was claimed earlier by a
// block that is running or done and waits on nothing later: the block waits
// (bounded) for the parent's flag, shifts the parent's local expansion into the
// cell and publishes its own flag.  A wait that gives up fills the cell's
// expansion with NaN, so the failure shows in the output.  ctl[0] (the claim
// counter) and the flags ctl[1 + c] start at zero.
__global__ void __launch_bounds__(128)
k_downward(int64_t nc, const int32_t *parent, const double *centre, DevTables tb, double *L,
           unsigned *ctl)
{
    extern __shared__ double sm[];
    __shared__ int s_c, s_ok;
    if (threadIdx.x == 0) s_c = (int)atomicAdd(&ctl[0], 1u);
    __syncthreads();
    const int c = s_c;
    if (c >= nc) return;
    const int pa = parent[c];
    if (pa >= 0) {
        if (threadIdx.x == 0) {
            s_ok = wait_flag(ctl + 1 + pa);
            __threadfence();
        }
        __syncthreads();
        if (s_ok) {
            l2l_cell(c, pa, centre, tb, L, sm);
        } else {
            for (int r = threadIdx.x; r < tb.nLh; r += blockDim.x)
                L[(int64_t)c * tb.nLh + r] = __longlong_as_double(0x7ff8000000000000ll);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicExch(ctl + 1 + c, 1u);
    }
}

}  // namespace

inline unsigned grid(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Table buffer layout (int32): lut | p2m | m2m_off | m2m_k | m2m_q | l2l_off |
// l2l_k | l2l_q | l2p_grad | red_off | red_src
fmm_status upload_tables(fmm_tree *t, int s, int p, int n_lo, DevTables *dt, const int32_t **lut)
{
    static int consts_ready[64] = {0};
    static std::mutex consts_mu;
    std::lock_guard<std::mutex> consts_lock(consts_mu);
    if (t->device < 64 && !consts_ready[t->device]) {
        const MultiIndex &I = multi_index();
        int8_t x[kMaxTot], y[kMaxTot], z[kMaxTot];
        for (int i = 0; i < kMaxTot; ++i) { x[i] = (int8_t)I.nx[i]; y[i] = (int8_t)I.ny[i]; z[i] = (int8_t)I.nz[i]; }
        FMM_TRY(cuda_check(t, cudaMemcpyToSymbol(c_nx, x, sizeof(x)), "constants"));
        FMM_TRY(cuda_check(t, cudaMemcpyToSymbol(c_ny, y, sizeof(y)), "constants"));
        FMM_TRY(cuda_check(t, cudaMemcpyToSymbol(c_nz, z, sizeof(z)), "constants"));
        double inv[kMaxOrder + 2];
        inv[0] = 0.0;
        for (int q = 1; q < kMaxOrder + 2; ++q) inv[q] = 1.0 / q;
        FMM_TRY(cuda_check(t, cudaMemcpyToSymbol(c_invint, inv, sizeof(inv)), "constants"));
        consts_ready[t->device] = 1;
    }
    OpTables &T = t->tab;
    std::vector<int32_t> buf;
    size_t o_lut, o_p2m, o_m2m_off, o_m2m_k, o_m2m_q, o_l2l_off, o_l2l_k, o_l2l_q, o_grad, o_roff, o_rsrc;
    auto put = [&](const std::vector<int> &v) {
        size_t o = buf.size();
        buf.insert(buf.end(), v.begin(), v.end());
        buf.push_back(0);
        return o;
    };
    const int h = t->m2l_harmonic ? 1 : 0;
    const int s_hi = std::max(s, t->s_hi);
    const bool rebuild = !(t->tab_key_s == s && t->tab_key_p == p && t->tab_key_nlo == n_lo &&
                           t->tab_key_h == h && t->tab_key_shi == s_hi);
    if (rebuild) build_tables(T, s, s_hi, p, n_lo, kM2LThreadsShared, h != 0);
    {
        const MultiIndex &I = multi_index();
        std::vector<int> lutv((kMaxOrder + 1) * (kMaxOrder + 1) * (kMaxOrder + 1));
        for (int i = 0; i < (int)lutv.size(); ++i) lutv[i] = ((const int16_t *)I.lut)[i];
        o_lut = put(lutv);
    }
    o_p2m = put(T.p2m_terms); o_m2m_off = put(T.m2m_off); o_m2m_k = put(T.m2m_k);
    o_m2m_q = put(T.m2m_q); o_l2l_off = put(T.l2l_off); o_l2l_k = put(T.l2l_k);
    o_l2l_q = put(T.l2l_q); o_grad = put(T.l2p_grad); o_roff = put(T.m2l_red_off);
    o_rsrc = put(T.m2l_red_src);
    const size_t o_hrm = put(T.h_rm), o_hf = put(T.h_fold), o_hfo = put(T.h_fold_off);
    const size_t o_hu = put(T.h_unfold), o_huo = put(T.h_unfold_off), o_hrn = put(T.h_rn);
    size_t o_mi;
    {
        const MultiIndex &I = multi_index();
        std::vector<int> mi(kMaxTot);
        for (int i = 0; i < kMaxTot; ++i)
            mi[i] = I.nx[i] | I.ny[i] << 5 | I.nz[i] << 10 | (I.nx[i] + I.ny[i] + I.nz[i]) << 15;
        o_mi = put(mi);
    }
    FMM_TRY(ensure(t, t->b_tab_i32, 4 * buf.size()));
    FMM_TRY(ensure(t, t->b_tab_u32, 4 * (T.m2l_desc.size() + 2)));
    if (rebuild) {
        FMM_TRY(cuda_check(t, cudaMemcpyAsync(t->b_tab_i32.ptr, buf.data(), 4 * buf.size(),
                                              cudaMemcpyHostToDevice, t->stream), "tables"));
        FMM_TRY(cuda_check(t, cudaMemcpyAsync(t->b_tab_u32.ptr, T.m2l_desc.data(),
                                              4 * T.m2l_desc.size(), cudaMemcpyHostToDevice,
                                              t->stream), "tables"));
        t->tab_key_s = s; t->tab_key_p = p; t->tab_key_nlo = n_lo; t->tab_key_h = h;
        t->tab_key_shi = s_hi;
    }
    const int32_t *B = (const int32_t *)t->b_tab_i32.ptr;
    dt->s = s; dt->p = p; dt->n_lo = n_lo; dt->nS = T.nS; dt->nM = T.nM; dt->nL = T.nL;
    dt->nD = T.nD; dt->m0 = T.m0; dt->nK = ntot(p); dt->nG = ntot(p - 1);
    dt->p2m_terms = B + o_p2m; dt->m2m_off = B + o_m2m_off; dt->m2m_k = B + o_m2m_k;
    dt->m2m_q = B + o_m2m_q; dt->l2l_off = B + o_l2l_off; dt->l2l_k = B + o_l2l_k;
    dt->l2l_q = B + o_l2l_q; dt->l2p_grad = B + o_grad; dt->m2l_red_off = B + o_roff;
    dt->m2l_red_src = B + o_rsrc;
    dt->m2l_desc = (const uint32_t *)t->b_tab_u32.ptr;
    dt->m2l_T = T.m2l_T; dt->m2l_slots = T.m2l_slots;
    dt->mi = B + o_mi;
    dt->harmonic = T.harmonic ? 1 : 0;
    dt->nMh = T.nMh;
    dt->h_fold_lev = (int)T.h_fold_off.size() - 1;
    dt->h_unfold_lev = (int)T.h_unfold_off.size() - 1;
    dt->h_rm = B + o_hrm; dt->h_fold = B + o_hf; dt->h_fold_off = B + o_hfo;
    dt->h_unfold = B + o_hu; dt->h_unfold_off = B + o_huo;
    dt->nLh = T.nLh; dt->h_rn = B + o_hrn;
    *lut = B + o_lut;
    return FMM_OK;
}

namespace {

void record(fmm_tree *t, int i)
{
    if (t->profiling) cudaEventRecord(t->ev[i], t->stream);
}

}  // namespace

void launch_fold_m(cudaStream_t st, const double *M, int ldM, int64_t nc, const DevTables &tb,
                   double *Mh, int ldH)
{
    if (nc > 0)
        k_fold_m<double><<<(unsigned)((nc + 3) / 4), 128, 32 * (size_t)tb.nM, st>>>(M, ldM, nc, tb, Mh, ldH);
}

void launch_fold_m(cudaStream_t st, const float *M, int ldM, int64_t nc, const DevTables &tb,
                   float *Mh, int ldH)
{
    if (nc > 0)
        k_fold_m<float><<<(unsigned)((nc + 3) / 4), 128, 32 * (size_t)tb.nM, st>>>(M, ldM, nc, tb, Mh, ldH);
}

// derivative tables, one FP64 row per distinct M2L offset key
fmm_status build_dtables(fmm_tree *t, int p, const DevTables &tb, const int32_t *lut)
{
    if (t->d_p != p && t->n_doff > 0) {
        FMM_TRY(ensure(t, t->b_D, 8 * (size_t)t->n_doff * tb.nD));
        // warps per block: as many rows of nD doubles as fit in 48 KB, at most 8
        const int wpb = (int)std::max<int64_t>(1, std::min<int64_t>(8, 49152 / (8 * (int64_t)tb.nD)));
        k_dtables<<<(unsigned)((t->n_doff + wpb - 1) / wpb), 32 * wpb, 8 * (size_t)wpb * tb.nD,
                    t->stream>>>((const uint64_t *)t->b_dkeys.ptr, t->n_doff, tb.nD, lut,
                                 (double *)t->b_D.ptr);
        ++t->launches;
        t->d_p = p;
        t->d32_p = -1;
        t->tc_img_p = -1;
        t->m32_img_p = -1;
    }
    return FMM_OK;
}

// P2M at the leaves and M2M upward, level by level, into b_M (FP64, tb.nM per cell)
fmm_status run_upward(fmm_tree *t, const DevTables &tb, bool rec)
{
    cudaStream_t st = t->stream;
    const int64_t nc = t->ncells;
    const int P1 = tb.p + 1;
    FMM_TRY(ensure(t, t->b_M, 8 * (size_t)nc * tb.nM));
    FMM_TRY(ensure(t, t->b_ud, 8 * (size_t)(nc + 1)));
    t->m_cells = nc;
    double *M = (double *)t->b_M.ptr;
    const double *centre = (const double *)t->b_centre.ptr;
    // P2M and M2M in one launch; the arrival counters start (and end) at zero
    cudaMemsetAsync(t->b_ud.ptr, 0, 4 * (size_t)nc, st);
    const size_t smem = 8 * std::max<size_t>(
        (size_t)kP2MChunk * 3 * P1 + (size_t)kP2MChunk * (tb.nK + 1) + (size_t)kP2MChunk * tb.nS,
        3 * (size_t)P1 + tb.nK + tb.nM);
    auto go = [&](auto kern) {
        allow_max_dynamic_smem(kern);
        kern<<<(unsigned)t->nleaves, kP2MThreads, smem, st>>>(
            (const int32_t *)t->b_leaves.ptr, (const int32_t *)t->b_begin.ptr,
            (const int32_t *)t->b_end.ptr, (const int32_t *)t->b_parent.ptr,
            (const int32_t *)t->b_child.ptr, (const int32_t *)t->b_nchild.ptr, centre,
            (const double *)t->b_px.ptr, (const double *)t->b_py.ptr, (const double *)t->b_pz.ptr,
            (const double *)t->b_S.ptr, tb, M, (unsigned *)t->b_ud.ptr);
    };
    if (tb.nS <= 3) go(k_upward<3>);
    else if (tb.nS <= 6) go(k_upward<6>);
    else go(k_upward<10>);
    ++t->launches;
    if (rec) record(t, 7);
    return FMM_OK;
}

fmm_status run_expansions(fmm_tree *t, int p, int want_phi, int want_field)
{
    cudaStream_t st = t->stream;
    const int s = t->s;
    const int n_lo = want_phi ? 0 : 1;
    DevTables tb;
    const int32_t *lut;
    FMM_TRY(upload_tables(t, s, p, n_lo, &tb, &lut));
    const int64_t nc = t->ncells, n = t->n;
    const int P1 = p + 1;

    FMM_TRY(build_dtables(t, p, tb, lut));
    record(t, 6);
    FMM_TRY(ensure(t, t->b_L, 8 * (size_t)nc * tb.nLh));
    FMM_TRY(ensure(t, t->b_phi, 8 * (size_t)n));
    FMM_TRY(ensure(t, t->b_E, 24 * (size_t)n));
    FMM_TRY(run_upward(t, tb, true));
    double *M = (double *)t->b_M.ptr, *L = (double *)t->b_L.ptr;
    const int32_t *leaves = (const int32_t *)t->b_leaves.ptr;
    const int32_t *begin = (const int32_t *)t->b_begin.ptr, *end = (const int32_t *)t->b_end.ptr;
    const double *centre = (const double *)t->b_centre.ptr;
    const double *px = (const double *)t->b_px.ptr, *py = (const double *)t->b_py.ptr,
                 *pz = (const double *)t->b_pz.ptr;
    // M2L over the stored lists (harmonic: on the folded multipoles)
    cudaMemsetAsync(L, 0, 8 * (size_t)nc * tb.nLh, st);
    const double *Ms = M;
    if (t->n_m2l > 0 && tb.harmonic) {
        FMM_TRY(ensure(t, t->b_Mh, 8 * (size_t)nc * tb.nMh));
        launch_fold_m(st, M, tb.nM, nc, tb, (double *)t->b_Mh.ptr, tb.nMh);
        ++t->launches;
        Ms = (const double *)t->b_Mh.ptr;
    }
    record(t, 8);
    if (t->n_m2l > 0) {
        const int ldM = tb.nMh | 1, ldD = tb.nD | 1;
        size_t fixed = 8 * (size_t)tb.m2l_slots * kM2LThreads + 4 * (size_t)tb.m2l_T * kM2LThreads;
        size_t smem = fixed + 8 * (size_t)kM2LBatch * (ldM + ldD);
        allow_max_dynamic_smem(k_m2l);
        k_m2l<<<(unsigned)nc, kM2LThreads, smem, st>>>(
            (const int32_t *)t->b_m2l_off.ptr, (const int32_t *)t->b_m2l_src.ptr,
            (const int32_t *)t->b_m2l_didx.ptr, (const int32_t *)t->b_level.ptr,
            (const int32_t *)t->b_sys.ptr, t->sys_eside_dev(), Ms, (const double *)t->b_D.ptr, tb, L);
        ++t->launches;
    }
    record(t, 9);
    // L2L downward, all levels in one launch (flags and claim counter start at zero)
    if (t->nlevels > 1) {
        unsigned *ctl = (unsigned *)t->b_ud.ptr + nc + 1;
        cudaMemsetAsync(ctl, 0, 4 * (size_t)(nc + 1), st);
        size_t smem = 8 * (size_t)(3 * P1 + tb.nK + tb.nL);
        k_downward<<<(unsigned)nc, 128, smem, st>>>(nc, (const int32_t *)t->b_parent.ptr, centre, tb, L, ctl);
        ++t->launches;
    }
    record(t, 10);
    // L2P
    {
        size_t smem = 8 * (size_t)(tb.nL + kL2PThreads * 3 * P1);
        allow_max_dynamic_smem(k_l2p);
        k_l2p<<<(unsigned)t->nleaves, kL2PThreads, smem, st>>>(leaves, begin, end, centre, px, py, pz,
                                                               L, tb, want_phi, want_field,
                                                               (double *)t->b_phi.ptr,
                                                               (double *)t->b_E.ptr);
        ++t->launches;
    }
    record(t, 11);
    return cuda_check(t, cudaGetLastError(), "expansion kernels");
}

}  // namespace fmm
