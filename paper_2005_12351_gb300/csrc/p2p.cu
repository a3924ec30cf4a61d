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

#include "fmm_internal.cuh"

namespace fmm {

namespace {

template <int S, bool PHI, bool FIELD>
__device__ __forceinline__ void pair_fp64(double dx, double dy, double dz, const double *Sj,
                                          double &f, double &e0, double &e1, double &e2)
{
    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double rinv = r2 > 0.0 ? rsqrt(r2) : 0.0;
    const double rinv2 = rinv * rinv;
    if (S == 0) {
        const double q = Sj[0];
        if (PHI) f = fma(q, rinv, f);
        if (FIELD) {
            const double w = q * rinv * rinv2;
            e0 = fma(w, dx, e0); e1 = fma(w, dy, e1); e2 = fma(w, dz, e2);
        }
    } else if (S == 1) {
        const double rinv3 = rinv * rinv2;
        const double sr = fma(Sj[0], dx, fma(Sj[1], dy, Sj[2] * dz));
        if (PHI) f = fma(-sr, rinv3, f);
        if (FIELD) {
            const double w = 3.0 * sr * rinv3 * rinv2;
            e0 = fma(Sj[0], rinv3, fma(-w, dx, e0));
            e1 = fma(Sj[1], rinv3, fma(-w, dy, e1));
            e2 = fma(Sj[2], rinv3, fma(-w, dz, e2));
        }
    } else {
        const double rinv3 = rinv * rinv2, rinv5 = rinv3 * rinv2;
        // half-gradient of q: h = (grad q)/2 is not symmetric in the S layout, so form grad q
        const double gq0 = fma(2.0 * Sj[0], dx, fma(Sj[1], dy, Sj[2] * dz));
        const double gq1 = fma(Sj[1], dx, fma(2.0 * Sj[3], dy, Sj[4] * dz));
        const double gq2 = fma(Sj[2], dx, fma(Sj[4], dy, 2.0 * Sj[5] * dz));
        // q = (R . grad q) / 2 for a homogeneous quadratic
        const double q = 0.5 * fma(gq0, dx, fma(gq1, dy, gq2 * dz));
        const double tr = Sj[0] + Sj[3] + Sj[5];
        if (PHI) f += 3.0 * q * rinv5 - tr * rinv3;
        if (FIELD) {
            const double a = 3.0 * rinv5;
            const double w = fma(15.0 * q, rinv5 * rinv2, -3.0 * tr * rinv5);
            e0 = fma(w, dx, fma(-a, gq0, e0));
            e1 = fma(w, dy, fma(-a, gq1, e1));
            e2 = fma(w, dz, fma(-a, gq2, e2));
        }
    }
}

constexpr int kP2PThreads = 128;

// One block per target leaf.  A leaf of nt <= 128 targets is covered
// floor(128/nt) times; each copy takes every k-th particle of every source
// leaf, and the copies are summed in a fixed order.  The block then adds the
// far field from L2P and writes phi, E at the caller's original index.
template <int S, bool PHI, bool FIELD>
__global__ void __launch_bounds__(kP2PThreads)
k_p2p(const int32_t *leaves, const int32_t *begin, const int32_t *end, const int32_t *off,
      const int32_t *src, const double *px, const double *py, const double *pz, const double *Sm,
      const double *phi_far, const double *E_far, const int32_t *perm, double *phi_out,
      double *E_out)
{
    constexpr int nS = (S + 1) * (S + 2) / 2;
    __shared__ double red[4][kP2PThreads];
    const int c = leaves[blockIdx.x];
    const int b = begin[c], e = end[c], nt = e - b;
    const int q0 = off[c], q1 = off[c + 1];
    const int tid = threadIdx.x;
    for (int t0 = 0; t0 < nt; t0 += kP2PThreads) {
        const int cnt = min(kP2PThreads, nt - t0);
        const int k = max(1, kP2PThreads / cnt);
        const int ti = tid % cnt, sp = tid / cnt;
        double f = 0.0, e0 = 0.0, e1 = 0.0, e2 = 0.0;
        if (sp < k) {
            const int i = b + t0 + ti;
            const double xi = px[i], yi = py[i], zi = pz[i];
            for (int q = q0; q < q1; ++q) {
                const int sl = src[q];
                const int je = end[sl];
                for (int j = begin[sl] + sp; j < je; j += k) {
                    double Sj[nS];
#pragma unroll
                    for (int a = 0; a < nS; ++a) Sj[a] = Sm[(int64_t)j * nS + a];
                    pair_fp64<S, PHI, FIELD>(xi - px[j], yi - py[j], zi - pz[j], Sj, f, e0, e1, e2);
                }
            }
        }
        red[0][tid] = f; red[1][tid] = e0; red[2][tid] = e1; red[3][tid] = e2;
        __syncthreads();
        if (tid < cnt) {
            for (int u = 1; u < k; ++u) {
                f += red[0][u * cnt + tid];
                e0 += red[1][u * cnt + tid];
                e1 += red[2][u * cnt + tid];
                e2 += red[3][u * cnt + tid];
            }
            const int i = b + t0 + tid;
            const int64_t o = perm[i];
            if (PHI) phi_out[o] = phi_far[i] + f;
            if (FIELD) {
                E_out[3 * o] = E_far[3 * (int64_t)i] + e0;
                E_out[3 * o + 1] = E_far[3 * (int64_t)i + 1] + e1;
                E_out[3 * o + 2] = E_far[3 * (int64_t)i + 2] + e2;
            }
        }
        __syncthreads();
    }
}

constexpr int kDirectThreads = 128;
constexpr int kDirectTile = 256;

template <int S, bool PHI, bool FIELD>
__global__ void __launch_bounds__(kDirectThreads)
k_direct(const double *pos, const double *mom, int64_t n, const int32_t *targets, int64_t nt,
         double *phi, double *E)
{
    constexpr int nS = (S + 1) * (S + 2) / 2;
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
                pair_fp64<S, PHI, FIELD>(xi - sx[u], yi - sy[u], zi - sz[u], sS + u * nS, f, e0,
                                         e1, e2);
    }
    if (t < nt) {
        if (!active) f = e0 = e1 = e2 = __longlong_as_double(0x7ff8000000000000ll);
        if (PHI) phi[t] = f;
        if (FIELD) { E[3 * t] = e0; E[3 * t + 1] = e1; E[3 * t + 2] = e2; }
    }
}

template <int S>
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
    if (want_phi && want_field) args(k_p2p<S, true, true>);
    else if (want_phi) args(k_p2p<S, true, false>);
    else args(k_p2p<S, false, true>);
}

template <int S>
void launch_direct_s(cudaStream_t st, const double *pos, const double *mom, int64_t n,
                     const int32_t *targets, int64_t nt, double *phi, double *E)
{
    const unsigned g = (unsigned)((nt + kDirectThreads - 1) / kDirectThreads);
    if (phi && E) k_direct<S, true, true><<<g, kDirectThreads, 0, st>>>(pos, mom, n, targets, nt, phi, E);
    else if (phi) k_direct<S, true, false><<<g, kDirectThreads, 0, st>>>(pos, mom, n, targets, nt, phi, E);
    else k_direct<S, false, true><<<g, kDirectThreads, 0, st>>>(pos, mom, n, targets, nt, phi, E);
}

}  // namespace

fmm_status run_p2p(fmm_tree *t, int want_phi, int want_field, double *phi_out, double *E_out)
{
    if (t->nleaves == 0) return FMM_OK;
    switch (t->s) {
    case 0: launch_p2p_s<0>(t, want_phi, want_field, phi_out, E_out); break;
    case 1: launch_p2p_s<1>(t, want_phi, want_field, phi_out, E_out); break;
    default: launch_p2p_s<2>(t, want_phi, want_field, phi_out, E_out); break;
    }
    ++t->launches;
    return cuda_check(t, cudaGetLastError(), "p2p kernel");
}

void launch_direct(cudaStream_t st, const double *pos, const double *mom, int64_t n, int s,
                   const int32_t *targets, int64_t nt, double *phi, double *E, int64_t *launches)
{
    if (nt <= 0 || (!phi && !E)) return;
    switch (s) {
    case 0: launch_direct_s<0>(st, pos, mom, n, targets, nt, phi, E); break;
    case 1: launch_direct_s<1>(st, pos, mom, n, targets, nt, phi, E); break;
    default: launch_direct_s<2>(st, pos, mom, n, targets, nt, phi, E); break;
    }
    ++*launches;
}

}  // namespace fmm
