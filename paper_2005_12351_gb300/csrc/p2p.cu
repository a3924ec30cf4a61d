// p2p.cu -- near field (P2P) and the FP64 direct sum.
//
// A source j seen from target i (paper §3.1 P2P operator, §2 Eq. (1)):
//   phi_i += sum_{|a|=s} S_{j,a} D_a(R),  E_i -= sum_a S_{j,a} grad D_a(R),  R = x_i - x_j,
// written out per source order:
//   s = 0:  phi = q/r,                       E = q R / r^3
//   s = 1:  phi = -(S.R)/r^3,                E = S/r^3 - 3 (S.R) R / r^5
//   s = 2:  phi = 3 q(R)/r^5 - tr/r^3,       E = -[3 grad q / r^5 - 15 q R / r^7 + 3 tr R / r^5]
//           with q(R) = sum_{|a|=2} S_a R^a and tr = S_200 + S_020 + S_002.
// Pairs with r = 0 (the target itself, coincident points) contribute nothing.
#include <algorithm>
#include <cstdlib>

#include "fmm_internal.cuh"
#include "pair.cuh"

namespace fmm {

namespace {

// 1/sqrt(x) for x > 0 in FP64 without the double-precision MUFU path:
//  1. x = m 4^k with m in [1, 4), by integer operations on the exponent;
//  2. an FP32 seed y_m = rsqrtf(m) (m rounded toward zero to float);
//  3. y0 = y_m 2^-k, assembled from the float's bits;
//  4. one third-order Householder step for f(y) = y^-2 - x:
//        e = 1 - x y0^2,   y = y0 + y0 e (1/2 + 3/8 e),
//     which leaves a relative error of about (5/16) e^3 ~ 2^-67 before the
//     final roundings (e ~ 2^-22 from the seed).  Five FP64 operations.
// x = 0 returns a finite value of no meaning (the callers mask r = 0).  A subnormal x (exponent field 0,
// x != 0: pairs closer than ~1.5e-154) takes CUDA's rsqrt instead: the
// exponent arithmetic above assumes a normal number.  The test is integer
// work only, so the FP64 pipe of the common path is unchanged.
__device__ __forceinline__ double rsqrt_hh(double x)
{
    const int hi = __double2hiint(x), lo = __double2loint(x);
    if (__builtin_expect((hi & 0x7ff00000) == 0 && (hi | lo) != 0, 0)) return rsqrt(x);
    const int ex = ((hi >> 20) & 0x7ff) - 1023;                 // unbiased exponent
    const int k = ex >> 1;                                      // floor(ex / 2)
    const int mhi = (hi & 0x000fffff) | ((1023 + (ex - 2 * k)) << 20);   // m in [1, 4)
    // float with m's exponent and the top 23 mantissa bits
    const int fbits = ((mhi - (896 << 20)) << 3) | ((unsigned)lo >> 29);
    const float ym = rsqrtf(__int_as_float(fbits));
    const int yb = __float_as_int(ym);
    const int yhi = ((yb >> 3) + (896 << 20)) - (k << 20);
    const double y0 = __hiloint2double(yhi, yb << 29);
    const double t = x * y0;
    const double e = fma(-t, y0, 1.0);
    const double c = fma(e, 0.375, 0.5);
    const double u = y0 * e;
    return fma(u, c, y0);
}

__global__ void k_check_rsqrt(const double *x, int64_t n, double *own, double *ref)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    own[i] = rsqrt_hh(x[i]);
    ref[i] = rsqrt(x[i]);
}

constexpr int kP2PThreads = 128;
constexpr int kP2PChunk = 512;            // source particles staged per round

// One source seen from one target, FP64, with S3 = 3 S pre-scaled in shared memory.
template <int S, bool PHI, bool FIELD>
__device__ __forceinline__ void pair_p2p(double dx, double dy, double dz, const double *Sj,
                                         const double *S3j, double &f, double &e0, double &e1,
                                         double &e2)
{
    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    // r2 >= 0, so "r2 > 0" is "its bit pattern is nonzero": an integer test
    const double y = __double_as_longlong(r2) != 0 ? rsqrt_hh(r2) : 0.0;
    const double y2 = y * y;
    if (S == 0) {
        if (PHI) f = fma(Sj[0], y, f);
        if (FIELD) {
            const double w = Sj[0] * (y * y2);
            e0 = fma(w, dx, e0); e1 = fma(w, dy, e1); e2 = fma(w, dz, e2);
        }
    } else if (S == 1) {
        const double y3 = y * y2;
        if (PHI) f = fma(-fma(Sj[0], dx, fma(Sj[1], dy, Sj[2] * dz)), y3, f);
        if (FIELD) {
            // E = S/r^3 - 3 (S.R) R / r^5
            const double w3 = fma(S3j[0], dx, fma(S3j[1], dy, S3j[2] * dz)) * (y3 * y2);
            e0 = fma(Sj[0], y3, fma(-w3, dx, e0));
            e1 = fma(Sj[1], y3, fma(-w3, dy, e1));
            e2 = fma(Sj[2], y3, fma(-w3, dz, e2));
        }
    } else {
        pair_fp64<2, PHI, FIELD>(dx, dy, dz, Sj, f, e0, e1, e2);
    }
}

// The partner leaves of one staging round, taken by warp 0 in parallel: lane l
// the list entry q + l (the first continues at particle j_in of its leaf); a
// prefix sum of their sizes decides which fit in cap particles (the last one
// possibly in part).  Writes groups [0, ng): first particle gbeg and offset
// gpre in the round, gpre[ng] = the round's size, and where the next round
// starts.  Requires q < q1.
__device__ __forceinline__ void stage_groups(int lane, int q, int q1, int j_in, int cap,
                                             const int32_t *src, const int32_t *begin,
                                             const int32_t *end, int *gbeg, int *gpre, int *ngroups,
                                             int *next_q, int *next_j)
{
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
    const bool in = qq < q1 && excl < cap;
    const int tk = in ? min(take, cap - excl) : 0;
    if (in) {
        gbeg[lane] = lb;
        gpre[lane] = excl;
    }
    const int ng = __popc(__ballot_sync(0xffffffffu, in));   // the taken entries: a prefix
    if (lane == ng - 1) {
        const bool whole = tk == take;
        gpre[ng] = excl + tk;
        *ngroups = ng;
        *next_q = whole ? qq + 1 : qq;
        *next_j = whole ? 0 : (lb - begin[sl]) + tk;
    }
}

// One block per target leaf.  The flattened source list of the leaf (all
// particles of its P2P partner leaves, in list order) is staged in shared
// memory in rounds of up to kP2PChunk particles from at most 32 leaves.  A leaf of nt <= 128 targets is covered k = floor(128/nt) times and
// copy c takes the staged sources c, c+k, c+2k, ..., so all threads run the
// same trip count.  Copies are combined in a fixed order, the L2P far field
// is added and the result is written at the caller's original index.
constexpr int kP2PGroups = 64;

template <int S, bool PHI, bool FIELD>
__global__ void __launch_bounds__(kP2PThreads)
k_p2p(const int32_t *leaves, const int32_t *begin, const int32_t *end, const int32_t *off,
      const int32_t *src, const double *px, const double *py, const double *pz, const double *Sm,
      const double *phi_far, const double *E_far, const int32_t *perm, double *phi_out,
      double *E_out)
{
    constexpr int nS = (S + 1) * (S + 2) / 2;
    __shared__ double sx[kP2PChunk], sy[kP2PChunk], sz[kP2PChunk];
    __shared__ double sS[kP2PChunk * nS], sS3[S == 1 ? kP2PChunk * 3 : 1];
    __shared__ double red[4][kP2PThreads];
    __shared__ int gbeg[kP2PGroups], gpre[kP2PGroups + 1];
    __shared__ int s_next_q, s_next_j, s_ngroups;
    const int c = leaves[blockIdx.x];
    const int b = begin[c], e = end[c], nt = e - b;
    const int q0 = off[c], q1 = off[c + 1];
    const int tid = threadIdx.x;
    for (int t0 = 0; t0 < nt; t0 += kP2PThreads) {
        const int cnt = min(kP2PThreads, nt - t0);
        const int k = max(1, kP2PThreads / cnt);
        const int ti = tid % cnt, sp = tid / cnt;
        const bool act = sp < k;
        const int i = b + t0 + ti;
        const double xi = act ? px[i] : 0.0, yi = act ? py[i] : 0.0, zi = act ? pz[i] : 0.0;
        double f = 0.0, e0 = 0.0, e1 = 0.0, e2 = 0.0;
        int q = q0, j_in = 0;                 // next partner leaf and offset inside it
        while (q < q1) {
            __syncthreads();                  // previous round's staged data is consumed
            if (tid < 32)
                stage_groups(tid, q, q1, j_in, kP2PChunk, src, begin, end, gbeg, gpre, &s_ngroups,
                             &s_next_q, &s_next_j);
            __syncthreads();
            const int ng = s_ngroups, used = gpre[ng];
            for (int d = tid; d < used; d += kP2PThreads) {
                int lo = 0, hi = ng - 1;      // last group with gpre[g] <= d
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (gpre[mid] <= d) lo = mid; else hi = mid - 1;
                }
                const int j = gbeg[lo] + (d - gpre[lo]);
                sx[d] = px[j]; sy[d] = py[j]; sz[d] = pz[j];
#pragma unroll
                for (int a = 0; a < nS; ++a) {
                    const double v = Sm[(int64_t)j * nS + a];
                    sS[d * nS + a] = v;
                    if (S == 1) sS3[d * 3 + a] = 3.0 * v;
                }
            }
            __syncthreads();
            if (act)
                for (int j = sp; j < used; j += k)
                    pair_p2p<S, PHI, FIELD>(xi - sx[j], yi - sy[j], zi - sz[j], sS + j * nS,
                                            S == 1 ? sS3 + j * 3 : sS, f, e0, e1, e2);
            q = s_next_q;
            j_in = s_next_j;
        }
        __syncthreads();
        red[0][tid] = f; red[1][tid] = e0; red[2][tid] = e1; red[3][tid] = e2;
        __syncthreads();
        if (tid < cnt) {
            for (int u = 1; u < k; ++u) {
                f += red[0][u * cnt + tid];
                e0 += red[1][u * cnt + tid];
                e1 += red[2][u * cnt + tid];
                e2 += red[3][u * cnt + tid];
            }
            const int ii = b + t0 + tid;
            const int64_t o = perm[ii];
            if (PHI) phi_out[o] = phi_far[ii] + f;
            if (FIELD) {
                E_out[3 * o] = E_far[3 * (int64_t)ii] + e0;
                E_out[3 * o + 1] = E_far[3 * (int64_t)ii + 1] + e1;
                E_out[3 * o + 2] = E_far[3 * (int64_t)ii + 2] + e2;
            }
        }
        __syncthreads();
    }
}

// Variant with two targets per thread: each staged source is read once from
// shared memory for two pair evaluations.  A chunk of up to 2*128 targets is
// split into halves of h = ceil(cnt/2); thread (ti, copy) owns targets ti and
// ti + h (the second one only if it exists).
// SHI > S: every particle carries the orders S..SHI (mixed systems), the pair
// terms summed shell by shell; fewer sources staged per round when the rows
// are wide.
template <int S, bool PHI, bool FIELD, int SHI = S>
__global__ void __launch_bounds__(kP2PThreads)
k_p2p_x2(const int32_t *leaves, const int32_t *begin, const int32_t *end, const int32_t *off,
         const int32_t *src, const double *px, const double *py, const double *pz,
         const double *Sm, const double *phi_far, const double *E_far, const int32_t *perm,
         double *phi_out, double *E_out)
{
    constexpr int nS = Orders<S, SHI>::n;
    constexpr bool kS3 = S == 1 && SHI == 1;           // 3 S staged for the dipole field
    constexpr int kP2PChunk = nS > 6 ? 256 : fmm::kP2PChunk;
    __shared__ double sx[kP2PChunk], sy[kP2PChunk], sz[kP2PChunk];
    __shared__ double sS[kP2PChunk * nS], sS3[kS3 ? kP2PChunk * 3 : 1];
    __shared__ double red[8][kP2PThreads];
    __shared__ int gbeg[kP2PGroups], gpre[kP2PGroups + 1];
    __shared__ int s_next_q, s_next_j, s_ngroups;
    const int c = leaves[blockIdx.x];
    const int b = begin[c], e = end[c], nt = e - b;
    const int q0 = off[c], q1 = off[c + 1];
    const int tid = threadIdx.x;
    for (int t0 = 0; t0 < nt; t0 += 2 * kP2PThreads) {
        const int cnt = min(2 * kP2PThreads, nt - t0);
        const int h = (cnt + 1) / 2;
        const int k = max(1, kP2PThreads / h);
        const int ti = tid % h, sp = tid / h;
        const bool act = sp < k;
        const bool two = act && (ti + h < cnt);
        const int i = b + t0 + ti, i2 = i + h;
        const double xi = act ? px[i] : 0.0, yi = act ? py[i] : 0.0, zi = act ? pz[i] : 0.0;
        const double xj = two ? px[i2] : 0.0, yj = two ? py[i2] : 0.0, zj = two ? pz[i2] : 0.0;
        double f = 0.0, e0 = 0.0, e1 = 0.0, e2 = 0.0;
        double g = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
        int q = q0, j_in = 0;
        while (q < q1) {
            __syncthreads();
            if (tid < 32)
                stage_groups(tid, q, q1, j_in, kP2PChunk, src, begin, end, gbeg, gpre, &s_ngroups,
                             &s_next_q, &s_next_j);
            __syncthreads();
            const int ng = s_ngroups, used = gpre[ng];
            for (int d = tid; d < used; d += kP2PThreads) {
                int lo = 0, hi = ng - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (gpre[mid] <= d) lo = mid; else hi = mid - 1;
                }
                const int j = gbeg[lo] + (d - gpre[lo]);
                sx[d] = px[j]; sy[d] = py[j]; sz[d] = pz[j];
#pragma unroll
                for (int a = 0; a < nS; ++a) {
                    const double v = Sm[(int64_t)j * nS + a];
                    sS[d * nS + a] = v;
                    if (kS3) sS3[d * 3 + a] = 3.0 * v;
                }
            }
            __syncthreads();
            if (act) {
                for (int j = sp; j < used; j += k) {
                    const double ax = sx[j], ay = sy[j], az = sz[j];
                    const double *Sj = sS + j * nS, *S3 = kS3 ? sS3 + j * 3 : sS;
                    if constexpr (SHI == S) {
                        pair_p2p<S, PHI, FIELD>(xi - ax, yi - ay, zi - az, Sj, S3, f, e0, e1, e2);
                        if (two) pair_p2p<S, PHI, FIELD>(xj - ax, yj - ay, zj - az, Sj, S3, g, g0, g1, g2);
                    } else {
                        pair_orders<S, SHI, PHI, FIELD>(xi - ax, yi - ay, zi - az, Sj, f, e0, e1, e2);
                        if (two) pair_orders<S, SHI, PHI, FIELD>(xj - ax, yj - ay, zj - az, Sj, g, g0, g1, g2);
                    }
                }
            }
            q = s_next_q;
            j_in = s_next_j;
        }
        __syncthreads();
        red[0][tid] = f; red[1][tid] = e0; red[2][tid] = e1; red[3][tid] = e2;
        red[4][tid] = g; red[5][tid] = g0; red[6][tid] = g1; red[7][tid] = g2;
        __syncthreads();
        if (tid < h) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                if (half == 1 && tid + h >= cnt) break;
                const int r = 4 * half;
                double F = red[r][tid], A = red[r + 1][tid], B = red[r + 2][tid], C = red[r + 3][tid];
                for (int u = 1; u < k; ++u) {
                    F += red[r][u * h + tid];
                    A += red[r + 1][u * h + tid];
                    B += red[r + 2][u * h + tid];
                    C += red[r + 3][u * h + tid];
                }
                const int ii = b + t0 + tid + half * h;
                const int64_t o = perm[ii];
                if (PHI) phi_out[o] = phi_far[ii] + F;
                if (FIELD) {
                    E_out[3 * o] = E_far[3 * (int64_t)ii] + A;
                    E_out[3 * o + 1] = E_far[3 * (int64_t)ii + 1] + B;
                    E_out[3 * o + 2] = E_far[3 * (int64_t)ii + 2] + C;
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ symmetric P2P
// Newton's third law in the near field.  The lists hold a leaf pair in both
// rows, (A, B) and (B, A), whenever the traversal reaches both orders (on the
// trees built here every pair of distinct leaves is mirrored), and the two
// directions of a particle pair share R = x_i - x_j up to sign, r^2, 1/r and
// its powers.  So A's block evaluates each mirrored pair with B > A once: the
// forward terms go to A's targets, the reverse terms to rows of B's particles
// in a buffer, and a second kernel adds, per target, the forward sum and the
// rows of its leaf's lower partners in list order, then the far field.  The
// reverse term of target j from source i is the forward formula with the
// moments of i and -R: by the parity of D_n (§2), the potential of an order-s
// source changes sign by (-1)^s under R -> -R and its field by (-1)^(s+1).
// Self entries (A, A) and entries without a mirror are evaluated forward only.
// A particle carrying the orders SLO..SHI (§2 mixed systems) takes the sum of
// its shells' terms in both directions, each shell with its own parity.
constexpr int kSymThreads = 128;
constexpr int kSymWarps = kSymThreads / 32;
constexpr int kSymTargets = 128;           // targets staged in shared memory per round

// Moment terms a pair reads: S itself for s <= 1; for s = 2 the entries of the
// (symmetric) gradient operator of q(R) = sum_{|a|=2} S_a R^a, i.e.
// (2 S_200, S_110, S_101, 2 S_020, S_011, 2 S_002), and the trace.
template <int S> struct SymMom { static constexpr int n = S == 2 ? 7 : (S + 1) * (S + 2) / 2; };

__host__ __device__ constexpr int sym_shell(int s) { return (s + 1) * (s + 2) / 2; }
__host__ __device__ constexpr int sym_terms(int s) { return s == 2 ? 7 : sym_shell(s); }
// offsets of shell s among the orders slo..: in the particle's moments, in the pair terms
__host__ __device__ constexpr int sym_shell_off(int slo, int s)
{
    return s <= slo ? 0 : sym_shell_off(slo, s - 1) + sym_shell(s - 1);
}
__host__ __device__ constexpr int sym_terms_off(int slo, int s)
{
    return s <= slo ? 0 : sym_terms_off(slo, s - 1) + sym_terms(s - 1);
}
template <int SLO, int SHI> struct SymMomOrders { static constexpr int n = sym_terms_off(SLO, SHI + 1); };

template <int S>
__device__ __forceinline__ void sym_load_mom(const double *Sj, double *m)
{
    if (S < 2) {
#pragma unroll
        for (int a = 0; a < (S + 1) * (S + 2) / 2; ++a) m[a] = Sj[a];
    } else {
        const double s0 = Sj[0], s1 = Sj[1], s2 = Sj[2], s3 = Sj[3], s4 = Sj[4], s5 = Sj[5];
        m[0] = 2.0 * s0; m[1] = s1; m[2] = s2; m[3] = 2.0 * s3; m[4] = s4; m[5] = 2.0 * s5;
        m[6] = s0 + s3 + s5;
    }
}

template <int SLO, int SHI>
__device__ __forceinline__ void sym_load_orders(const double *Sj, double *m)
{
    sym_load_mom<SLO>(Sj, m);
    if constexpr (SHI >= SLO + 1)
        sym_load_mom<SLO + 1>(Sj + sym_shell_off(SLO, SLO + 1), m + sym_terms_off(SLO, SLO + 1));
    if constexpr (SHI >= SLO + 2)
        sym_load_mom<SLO + 2>(Sj + sym_shell_off(SLO, SLO + 2), m + sym_terms_off(SLO, SLO + 2));
}

// The part of a pair both directions share (for the orders SLO..SHI).
struct SymGeo {
    double dx, dy, dz, y, y3, a1, c1, c2, c3;
};

template <int SLO, int SHI, bool PHI, bool FIELD>
__device__ __forceinline__ SymGeo sym_geo(double dx, double dy, double dz)
{
    SymGeo g;
    g.dx = dx; g.dy = dy; g.dz = dz;
    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    g.y = __double_as_longlong(r2) != 0 ? rsqrt_hh(r2) : 0.0;
    const double y2 = g.y * g.y;
    g.y3 = g.y * y2;
    g.a1 = g.c1 = g.c2 = g.c3 = 0.0;
    if (SLO <= 1 && SHI >= 1 && FIELD) g.a1 = 3.0 * y2;  // 3 / r^2 (dipole field)
    if (SHI == 2) {
        const double y5 = g.y3 * y2;
        g.c1 = 3.0 * y5;                                 // 3 / r^5
        if (PHI) g.c2 = 1.5 * y5;
        if (FIELD) g.c3 = 7.5 * (y5 * y2);               // 15 / (2 r^7)
    }
    return g;
}

// One direction of a pair into the accumulators a = ([phi], [E_x, E_y, E_z]):
// forward (target i, source moments m of j) or, with REV, reverse (target j,
// source moments m of i).  Same formulas as pair_fp64 with R -> -R for REV.
template <int S, bool PHI, bool FIELD, bool REV>
__device__ __forceinline__ void sym_dir(const SymGeo &g, const double *m, double *a)
{
    constexpr int e = PHI ? 1 : 0;
    if (S == 0) {
        if (PHI) a[0] = fma(m[0], g.y, a[0]);
        if (FIELD) {
            const double w = REV ? -(m[0] * g.y3) : m[0] * g.y3;
            a[e] = fma(w, g.dx, a[e]);
            a[e + 1] = fma(w, g.dy, a[e + 1]);
            a[e + 2] = fma(w, g.dz, a[e + 2]);
        }
    } else if (S == 1) {
        const double sr = fma(m[0], g.dx, fma(m[1], g.dy, m[2] * g.dz));
        if (PHI) a[0] = fma(REV ? sr : -sr, g.y3, a[0]);
        if (FIELD) {
            // E = (S - 3 (S.R) R / r^2) / r^3, even in R
            const double v = sr * g.a1;
            a[e] = fma(fma(-v, g.dx, m[0]), g.y3, a[e]);
            a[e + 1] = fma(fma(-v, g.dy, m[1]), g.y3, a[e + 1]);
            a[e + 2] = fma(fma(-v, g.dz, m[2]), g.y3, a[e + 2]);
        }
    } else {
        const double gq0 = fma(m[0], g.dx, fma(m[1], g.dy, m[2] * g.dz));
        const double gq1 = fma(m[1], g.dx, fma(m[3], g.dy, m[4] * g.dz));
        const double gq2 = fma(m[2], g.dx, fma(m[4], g.dy, m[5] * g.dz));
        const double q2 = fma(gq0, g.dx, fma(gq1, g.dy, gq2 * g.dz));   // 2 q(R)
        const double tr = m[6];
        if (PHI) a[0] = fma(q2, g.c2, fma(-tr, g.y3, a[0]));             // 3q/r^5 - tr/r^3
        if (FIELD) {
            const double w = fma(q2, g.c3, -tr * g.c1);                  // 15q/r^7 - 3tr/r^5
            const double wa = REV ? -w : w, ca = REV ? g.c1 : -g.c1;
            a[e] = fma(wa, g.dx, fma(ca, gq0, a[e]));
            a[e + 1] = fma(wa, g.dy, fma(ca, gq1, a[e + 1]));
            a[e + 2] = fma(wa, g.dz, fma(ca, gq2, a[e + 2]));
        }
    }
}

// Both directions' shells of a mixed-order pair, the shells in ascending order.
template <int SLO, int SHI, bool PHI, bool FIELD, bool REV>
__device__ __forceinline__ void sym_dir_orders(const SymGeo &g, const double *m, double *a)
{
    sym_dir<SLO, PHI, FIELD, REV>(g, m, a);
    if constexpr (SHI >= SLO + 1)
        sym_dir<SLO + 1, PHI, FIELD, REV>(g, m + sym_terms_off(SLO, SLO + 1), a);
    if constexpr (SHI >= SLO + 2)
        sym_dir<SLO + 2, PHI, FIELD, REV>(g, m + sym_terms_off(SLO, SLO + 2), a);
}

// Warp totals of four partial sums: lanes 8c .. 8c+7 end with the total of
// v_c.  Two exchanges halve the vector, three more finish one value, in a
// fixed pattern (six additions per lane instead of twenty).
__device__ __forceinline__ double sym_warp_sum4(double v0, double v1, double v2, double v3)
{
    const int lane = threadIdx.x & 31;
    const bool h16 = lane & 16, h8 = lane & 8;
    double a = h16 ? v2 : v0, b = h16 ? v3 : v1;
    const double sa = h16 ? v0 : v2, sb = h16 ? v1 : v3;
    a += __shfl_xor_sync(0xffffffffu, sa, 16);
    b += __shfl_xor_sync(0xffffffffu, sb, 16);
    double c = h8 ? b : a;
    const double sc = h8 ? a : b;
    c += __shfl_xor_sync(0xffffffffu, sc, 8);
    c += __shfl_xor_sync(0xffffffffu, c, 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

__device__ __forceinline__ double sym_warp_sum1(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One batch of sources against the staged targets.  Thread tid holds the
// sources d0 + u*kSymThreads + tid (u < TJ) of the segment in registers and
// loops over the targets; the forward terms of each target are summed over
// the warp and added to the warp's row fw; with REV the reverse terms of the
// held sources are accumulated over all targets and stored to (first target
// round) or added to their rows of rev.
template <int S, bool PHI, bool FIELD, bool REV, int TJ, int SHI>
__device__ __forceinline__ void sym_batch(int d0, int used, int ne, const int *seg_q,
                                          const int *seg_pre, const int32_t *src,
                                          const int32_t *begin, const uint32_t *rbase,
                                          const double *px, const double *py, const double *pz,
                                          const double *Sm, const double *tx, const double *ty,
                                          const double *tz, const double *tm, int cntT,
                                          double (*fw)[4], double *rev, bool first)
{
    constexpr int nS = Orders<S, SHI>::n;
    constexpr int nM = SymMomOrders<S, SHI>::n;
    constexpr int NC = (PHI ? 1 : 0) + (FIELD ? 3 : 0);
    const int tid = threadIdx.x, lane = tid & 31;
    double sx[TJ], sy[TJ], sz[TJ], sm[TJ][nM], acc[TJ][NC];
    int64_t row[TJ];
    bool val[TJ];
#pragma unroll
    for (int u = 0; u < TJ; ++u) {
        const int d = d0 + u * kSymThreads + tid;
        val[u] = d < used;
        sx[u] = sy[u] = sz[u] = 0.0;
#pragma unroll
        for (int a = 0; a < nM; ++a) sm[u][a] = 0.0;
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[u][c] = 0.0;
        row[u] = 0;
        if (val[u]) {
            int lo = 0, hi = ne - 1;          // last entry with seg_pre <= d
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (seg_pre[mid] <= d) lo = mid; else hi = mid - 1;
            }
            const int q = seg_q[lo], k = d - seg_pre[lo];
            const int j = begin[src[q]] + k;
            sx[u] = px[j]; sy[u] = py[j]; sz[u] = pz[j];
            sym_load_orders<S, SHI>(Sm + (int64_t)j * nS, sm[u]);
            if (REV) row[u] = (int64_t)rbase[q] + k;
        }
    }
    for (int i = 0; i < cntT; ++i) {
        const double xi = tx[i], yi = ty[i], zi = tz[i];
        double mi[nM];
#pragma unroll
        for (int a = 0; a < nM; ++a) mi[a] = REV ? tm[i * nM + a] : 0.0;
        double f[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int u = 0; u < TJ; ++u) {
            if (!val[u]) continue;
            const SymGeo g = sym_geo<S, SHI, PHI, FIELD>(xi - sx[u], yi - sy[u], zi - sz[u]);
            sym_dir_orders<S, SHI, PHI, FIELD, false>(g, sm[u], f);
            if (REV) sym_dir_orders<S, SHI, PHI, FIELD, true>(g, mi, acc[u]);
        }
        if (NC == 1) {
            const double v = sym_warp_sum1(f[0]);
            if (lane == 0) fw[i][0] += v;
        } else {
            const double v = sym_warp_sum4(f[0], f[1], f[2], NC == 4 ? f[3] : 0.0);
            if ((lane & 7) == 0 && (lane >> 3) < NC) fw[i][lane >> 3] += v;
        }
    }
    if (REV) {
#pragma unroll
        for (int u = 0; u < TJ; ++u) {
            if (!val[u]) continue;
            double *r = rev + row[u] * NC;
#pragma unroll
            for (int c = 0; c < NC; ++c) r[c] = first ? acc[u][c] : r[c] + acc[u][c];
        }
    }
}

// One block per target leaf A.  For each round of up to kSymTargets staged
// targets: pass 0 takes the mirrored entries (A, B) with B > A (both
// directions), pass 1 the forward-only entries; each pass walks A's row in
// segments of 32 entries, compacted by warp 0 in list order.  The forward sum
// of a target is the warps' rows added in warp order.
template <int S, bool PHI, bool FIELD, int SHI = S>
__global__ void __launch_bounds__(kSymThreads)
k_p2p_sym(const int32_t *leaves, const int32_t *begin, const int32_t *end, const int32_t *off,
          const int32_t *src, const int32_t *mir, const uint32_t *rbase, const double *px,
          const double *py, const double *pz, const double *Sm, double *rev, double *fwd)
{
    constexpr int nS = Orders<S, SHI>::n;
    constexpr int nM = SymMomOrders<S, SHI>::n;
    constexpr int NC = (PHI ? 1 : 0) + (FIELD ? 3 : 0);
    constexpr int TJ = nM > 4 ? 2 : 4;       // sources per thread held in registers
    __shared__ double tx[kSymTargets], ty[kSymTargets], tz[kSymTargets], tm[kSymTargets * nM];
    __shared__ double fw[kSymWarps][kSymTargets][4];
    __shared__ int seg_q[32], seg_pre[33];
    __shared__ int s_ne;
    const int A = leaves[blockIdx.x];
    const int b = begin[A], nA = end[A] - b;
    const int q0 = off[A], q1 = off[A + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // a leaf without particles still runs one round: its partners' reverse rows are zero
    for (int t0 = 0; t0 == 0 || t0 < nA; t0 += kSymTargets) {
        const int cntT = max(0, min(kSymTargets, nA - t0));
        __syncthreads();
        for (int u = tid; u < cntT; u += kSymThreads) {
            const int i = b + t0 + u;
            tx[u] = px[i]; ty[u] = py[i]; tz[u] = pz[i];
            sym_load_orders<S, SHI>(Sm + (int64_t)i * nS, tm + u * nM);
        }
        for (int u = tid; u < kSymWarps * kSymTargets * 4; u += kSymThreads) (&fw[0][0][0])[u] = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
            for (int qs = q0; qs < q1; qs += 32) {
                __syncthreads();
                if (warp == 0) {
                    const int q = qs + lane;
                    int n = 0, take = 0;
                    if (q < q1) {
                        const int B = src[q], m = mir[q];
                        take = pass == 0 ? (m >= 0 && B > A) : (B == A || m < 0);
                        if (take) n = end[B] - begin[B];
                    }
                    int k = take, c = n;             // inclusive scans over the lanes
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int yk = __shfl_up_sync(0xffffffffu, k, o);
                        const int yc = __shfl_up_sync(0xffffffffu, c, o);
                        if (lane >= o) { k += yk; c += yc; }
                    }
                    if (take) { seg_q[k - 1] = q; seg_pre[k - 1] = c - n; }
                    if (lane == 31) { s_ne = k; seg_pre[k] = c; }
                }
                __syncthreads();
                const int ne = s_ne, used = seg_pre[ne];
                for (int d0 = 0; d0 < used; d0 += kSymThreads * TJ) {
                    if (pass == 0)
                        sym_batch<S, PHI, FIELD, true, TJ, SHI>(d0, used, ne, seg_q, seg_pre, src, begin,
                                                           rbase, px, py, pz, Sm, tx, ty, tz, tm,
                                                           cntT, fw[warp], rev, t0 == 0);
                    else
                        sym_batch<S, PHI, FIELD, false, TJ, SHI>(d0, used, ne, seg_q, seg_pre, src,
                                                            begin, rbase, px, py, pz, Sm, tx, ty,
                                                            tz, tm, cntT, fw[warp], rev, false);
                }
            }
        }
        __syncthreads();
        for (int u = tid; u < cntT; u += kSymThreads) {
            const int64_t i = b + t0 + u;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                double v = fw[0][u][c];
#pragma unroll
                for (int w = 1; w < kSymWarps; ++w) v += fw[w][u][c];
                fwd[i * NC + c] = v;
            }
        }
    }
}

// Per target of leaf A: the forward sum, then the reverse rows of each
// mirrored entry (A, B) with B < A in list order, then the far field; the
// result is written at the caller's original index.
template <bool PHI, bool FIELD>
__global__ void __launch_bounds__(kSymThreads)
k_p2p_sym_gather(const int32_t *leaves, const int32_t *begin, const int32_t *end,
                 const int32_t *off, const int32_t *src, const int32_t *mir,
                 const uint32_t *rbase, const double *rev, const double *fwd,
                 const double *phi_far, const double *E_far, const int32_t *perm,
                 double *phi_out, double *E_out)
{
    constexpr int NC = (PHI ? 1 : 0) + (FIELD ? 3 : 0);
    constexpr int e = PHI ? 1 : 0;
    const int A = leaves[blockIdx.x];
    const int b = begin[A], nA = end[A] - b;
    const int q0 = off[A], q1 = off[A + 1];
    for (int u = threadIdx.x; u < nA; u += kSymThreads) {
        const int64_t i = b + u;
        double v[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = fwd[i * NC + c];
        for (int q = q0; q < q1; ++q) {
            const int B = src[q], m = mir[q];
            if (m < 0 || B >= A) continue;
            const double *r = rev + ((int64_t)rbase[m] + u) * NC;
#pragma unroll
            for (int c = 0; c < NC; ++c) v[c] += r[c];
        }
        const int64_t o = perm[i];
        if (PHI) phi_out[o] = phi_far[i] + v[0];
        if (FIELD) {
            E_out[3 * o] = E_far[3 * i] + v[e];
            E_out[3 * o + 1] = E_far[3 * i + 1] + v[e + 1];
            E_out[3 * o + 2] = E_far[3 * i + 2] + v[e + 2];
        }
    }
}

// Plan, one thread per leaf A: for each entry (A, B) of A's row its mirror
// (B, A) in B's row (rows are sorted by source cell: binary search), -1 if
// none or B == A; cnt = |B| for mirrored entries with B > A, else 0; the
// 64-bit total of cnt.
__global__ void k_sym_plan(const int32_t *leaves, int64_t nleaves, const int32_t *begin,
                           const int32_t *end, const int32_t *off, const int32_t *src,
                           int32_t *mir, uint32_t *cnt, unsigned long long *total)
{
    const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long tot = 0;
    if (l < nleaves) {
        const int A = leaves[l];
        for (int q = off[A]; q < off[A + 1]; ++q) {
            const int B = src[q];
            int m = -1;
            if (B != A) {
                int lo = off[B], hi = off[B + 1];
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (src[mid] < A) lo = mid + 1; else hi = mid;
                }
                if (lo < off[B + 1] && src[lo] == A) m = lo;
            }
            mir[q] = m;
            const uint32_t c = (m >= 0 && B > A) ? (uint32_t)(end[B] - begin[B]) : 0u;
            cnt[q] = c;
            tot += c;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(total, tot);
}

constexpr int kDirectThreads = 128;
constexpr int kDirectTile = 256;

template <int S, bool PHI, bool FIELD, int SHI = S>
__global__ void __launch_bounds__(kDirectThreads)
k_direct(const double *pos, const double *mom, int64_t n, const int32_t *targets, int64_t nt,
         double *phi, double *E)
{
    constexpr int nS = Orders<S, SHI>::n;
    __shared__ double sx[kDirectTile], sy[kDirectTile], sz[kDirectTile], sS[kDirectTile * nS];
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t i = t < nt ? (targets ? (int64_t)targets[t] : t) : 0;
    const bool in_range = i >= 0 && i < n;
    const bool active = t < nt && in_range;
    if (!in_range) i = 0;              // out-of-range target: outputs NaN, no access
    const double xi = active ? pos[3 * i] : 0.0, yi = active ? pos[3 * i + 1] : 0.0,
                 zi = active ? pos[3 * i + 2] : 0.0;
    double f = 0.0, e0 = 0.0, e1 = 0.0, e2 = 0.0;
    for (int64_t j0 = 0; j0 < n; j0 += kDirectTile) {
        const int cnt = (int)min((int64_t)kDirectTile, n - j0);
        __syncthreads();
        for (int u = threadIdx.x; u < cnt; u += blockDim.x) {
            sx[u] = pos[3 * (j0 + u)];
            sy[u] = pos[3 * (j0 + u) + 1];
            sz[u] = pos[3 * (j0 + u) + 2];
        }
        for (int u = threadIdx.x; u < cnt * nS; u += blockDim.x) sS[u] = mom[j0 * nS + u];
        __syncthreads();
        if (active)
            for (int u = 0; u < cnt; ++u)
                pair_orders<S, SHI, PHI, FIELD>(xi - sx[u], yi - sy[u], zi - sz[u], sS + u * nS, f,
                                                e0, e1, e2);
    }
    if (t < nt) {
        if (!active) f = e0 = e1 = e2 = __longlong_as_double(0x7ff8000000000000ll);
        if (PHI) phi[t] = f;
        if (FIELD) { E[3 * t] = e0; E[3 * t + 1] = e1; E[3 * t + 2] = e2; }
    }
}

template <int S, int SHI = S>
void launch_sym_s(fmm_tree *t, int want_phi, int want_field, double *phi, double *E)
{
    const unsigned g = (unsigned)t->nleaves;
    cudaStream_t st = t->stream;
    const int32_t *lv = (const int32_t *)t->b_leaves.ptr, *bg = (const int32_t *)t->b_begin.ptr,
                  *en = (const int32_t *)t->b_end.ptr, *of = (const int32_t *)t->b_p2p_off.ptr,
                  *sr = (const int32_t *)t->b_p2p_src.ptr, *mi = (const int32_t *)t->b_sym_mir.ptr;
    const uint32_t *rb = (const uint32_t *)t->b_sym_base.ptr;
    const double *px = (const double *)t->b_px.ptr, *py = (const double *)t->b_py.ptr,
                 *pz = (const double *)t->b_pz.ptr, *Sm = (const double *)t->b_S.ptr;
    double *rev = (double *)t->b_sym_rev.ptr, *fwd = (double *)t->b_sym_fwd.ptr;
    auto run = [&](auto kern, auto gath) {
        kern<<<g, kSymThreads, 0, st>>>(lv, bg, en, of, sr, mi, rb, px, py, pz, Sm, rev, fwd);
        gath<<<g, kSymThreads, 0, st>>>(lv, bg, en, of, sr, mi, rb, rev, fwd,
                                        (const double *)t->b_phi.ptr, (const double *)t->b_E.ptr,
                                        (const int32_t *)t->b_perm.ptr, phi, E);
    };
    if (want_phi && want_field) run(k_p2p_sym<S, true, true, SHI>, k_p2p_sym_gather<true, true>);
    else if (want_phi) run(k_p2p_sym<S, true, false, SHI>, k_p2p_sym_gather<true, false>);
    else run(k_p2p_sym<S, false, true, SHI>, k_p2p_sym_gather<false, true>);
}

template <int S, int SHI = S>
void launch_p2p_s(fmm_tree *t, int want_phi, int want_field, double *phi, double *E)
{
    auto args = [&](auto kern) {
        kern<<<(unsigned)t->nleaves, kP2PThreads, 0, t->stream>>>(
            (const int32_t *)t->b_leaves.ptr, (const int32_t *)t->b_begin.ptr,
            (const int32_t *)t->b_end.ptr, (const int32_t *)t->b_p2p_off.ptr,
            (const int32_t *)t->b_p2p_src.ptr, (const double *)t->b_px.ptr,
            (const double *)t->b_py.ptr, (const double *)t->b_pz.ptr, (const double *)t->b_S.ptr,
            (const double *)t->b_phi.ptr, (const double *)t->b_E.ptr,
            (const int32_t *)t->b_perm.ptr, phi, E);
    };
    if (t->p2p_variant >= 1 || SHI != S) {         // mixed orders: this kernel only
        if (want_phi && want_field) args(k_p2p_x2<S, true, true, SHI>);
        else if (want_phi) args(k_p2p_x2<S, true, false, SHI>);
        else args(k_p2p_x2<S, false, true, SHI>);
        return;
    }
    if (want_phi && want_field) args(k_p2p<S, true, true>);
    else if (want_phi) args(k_p2p<S, true, false>);
    else args(k_p2p<S, false, true>);
}

template <int S, int SHI = S>
void launch_direct_s(cudaStream_t st, const double *pos, const double *mom, int64_t n,
                     const int32_t *targets, int64_t nt, double *phi, double *E)
{
    const unsigned g = (unsigned)((nt + kDirectThreads - 1) / kDirectThreads);
    if (phi && E) k_direct<S, true, true, SHI><<<g, kDirectThreads, 0, st>>>(pos, mom, n, targets, nt, phi, E);
    else if (phi) k_direct<S, true, false, SHI><<<g, kDirectThreads, 0, st>>>(pos, mom, n, targets, nt, phi, E);
    else k_direct<S, false, true, SHI><<<g, kDirectThreads, 0, st>>>(pos, mom, n, targets, nt, phi, E);
}

}  // namespace

// The plan of the symmetric P2P (cached with the lists; one host sync when it
// is built) and its buffers for NC output components.  FMM_EBUDGET when the
// buffers do not fit the handle's budget.
fmm_status sym_prepare(fmm_tree *t, int NC)
{
    cudaStream_t st = t->stream;
    const int64_t np = std::max<int64_t>(t->n_p2p, 1);
    if (!t->sym_plan) {
        FMM_TRY(ensure(t, t->b_sym_mir, 4 * (size_t)np));
        FMM_TRY(ensure(t, t->b_sym_cnt, 4 * (size_t)np));
        FMM_TRY(ensure(t, t->b_sym_base, 4 * (size_t)np));
        FMM_TRY(ensure(t, t->b_sym_scan, scan_scratch_bytes(np)));
        FMM_TRY(ensure(t, t->b_sym_tot, 16));
        unsigned long long *tot = (unsigned long long *)t->b_sym_tot.ptr;
        FMM_TRY(cuda_check(t, cudaMemsetAsync(t->b_sym_mir.ptr, 0xff, 4 * (size_t)np, st), "memset"));
        FMM_TRY(cuda_check(t, cudaMemsetAsync(t->b_sym_cnt.ptr, 0, 4 * (size_t)np, st), "memset"));
        FMM_TRY(cuda_check(t, cudaMemsetAsync(tot, 0, 8, st), "memset"));
        k_sym_plan<<<(unsigned)((t->nleaves + 127) / 128), 128, 0, st>>>(
            (const int32_t *)t->b_leaves.ptr, t->nleaves, (const int32_t *)t->b_begin.ptr,
            (const int32_t *)t->b_end.ptr, (const int32_t *)t->b_p2p_off.ptr,
            (const int32_t *)t->b_p2p_src.ptr, (int32_t *)t->b_sym_mir.ptr,
            (uint32_t *)t->b_sym_cnt.ptr, tot);
        ++t->launches;
        exclusive_scan_u32((const uint32_t *)t->b_sym_cnt.ptr, (uint32_t *)t->b_sym_base.ptr, np,
                           (uint32_t *)t->b_sym_scan.ptr, st, &t->launches);
        unsigned long long rows = 0;
        FMM_TRY(cuda_check(t, cudaMemcpyAsync(&rows, tot, 8, cudaMemcpyDeviceToHost, st), "rows"));
        FMM_TRY(cuda_check(t, cudaStreamSynchronize(st), "sync"));
        t->sym_rows = rows >= (1ull << 32) ? -1 : (int64_t)rows;
        t->sym_plan = true;
    }
    if (t->sym_rows < 0) return FMM_OK;
    FMM_TRY(ensure(t, t->b_sym_rev, 8 * (size_t)NC * (size_t)std::max<int64_t>(t->sym_rows, 1)));
    return ensure(t, t->b_sym_fwd, 8 * (size_t)NC * (size_t)std::max<int64_t>(t->n, 1));
}

fmm_status run_p2p(fmm_tree *t, int want_phi, int want_field, double *phi_out, double *E_out)
{
    if (t->nleaves == 0) return FMM_OK;
    const int so = t->s * 3 + t->s_hi;                 // (lowest, highest) source order
    if (t->p2p_variant == 2) {
        const fmm_status ps = sym_prepare(t, (want_phi ? 1 : 0) + (want_field ? 3 : 0));
        if (ps == FMM_OK && t->sym_rows >= 0) {
            switch (so) {
            case 0: launch_sym_s<0>(t, want_phi, want_field, phi_out, E_out); break;
            case 1: launch_sym_s<0, 1>(t, want_phi, want_field, phi_out, E_out); break;
            case 2: launch_sym_s<0, 2>(t, want_phi, want_field, phi_out, E_out); break;
            case 4: launch_sym_s<1>(t, want_phi, want_field, phi_out, E_out); break;
            case 5: launch_sym_s<1, 2>(t, want_phi, want_field, phi_out, E_out); break;
            default: launch_sym_s<2>(t, want_phi, want_field, phi_out, E_out); break;
            }
            t->launches += 2;
            return cuda_check(t, cudaGetLastError(), "symmetric p2p kernels");
        }
        if (ps != FMM_OK && ps != FMM_EBUDGET) return ps;
        t->err.clear();               // over the budget or the row index: two targets per thread
    }
    if (t->s_hi != t->s) {                            // mixed orders: two targets per thread
        switch (so) {
        case 1: launch_p2p_s<0, 1>(t, want_phi, want_field, phi_out, E_out); break;
        case 2: launch_p2p_s<0, 2>(t, want_phi, want_field, phi_out, E_out); break;
        default: launch_p2p_s<1, 2>(t, want_phi, want_field, phi_out, E_out); break;
        }
        ++t->launches;
        return cuda_check(t, cudaGetLastError(), "p2p kernel");
    }
    switch (t->s) {
    case 0: launch_p2p_s<0>(t, want_phi, want_field, phi_out, E_out); break;
    case 1: launch_p2p_s<1>(t, want_phi, want_field, phi_out, E_out); break;
    default: launch_p2p_s<2>(t, want_phi, want_field, phi_out, E_out); break;
    }
    ++t->launches;
    return cuda_check(t, cudaGetLastError(), "p2p kernel");
}

void launch_check_rsqrt(cudaStream_t st, const double *x, int64_t n, double *own, double *ref)
{
    if (n > 0) k_check_rsqrt<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, n, own, ref);
}

void launch_direct(cudaStream_t st, const double *pos, const double *mom, int64_t n, int s,
                   int s_hi, const int32_t *targets, int64_t nt, double *phi, double *E,
                   int64_t *launches)
{
    if (nt <= 0 || (!phi && !E)) return;
    switch (s * 3 + s_hi) {
    case 0: launch_direct_s<0>(st, pos, mom, n, targets, nt, phi, E); break;
    case 1: launch_direct_s<0, 1>(st, pos, mom, n, targets, nt, phi, E); break;
    case 2: launch_direct_s<0, 2>(st, pos, mom, n, targets, nt, phi, E); break;
    case 4: launch_direct_s<1>(st, pos, mom, n, targets, nt, phi, E); break;
    case 5: launch_direct_s<1, 2>(st, pos, mom, n, targets, nt, phi, E); break;
    default: launch_direct_s<2>(st, pos, mom, n, targets, nt, phi, E); break;
    }
    ++*launches;
}

}  // namespace fmm
