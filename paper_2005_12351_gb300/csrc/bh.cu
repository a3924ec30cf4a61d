// bh.cu -- multipolar Barnes-Hut (§2 multipole potential; §3.2 Methods), FP64.
//
// Multipoles of order p (s <= |m| <= p: the P2M/M2M of the FMM storage at
// order p - s), then for every target a walk from its system's root: a cell
// with r_cell^2 < theta^2 |x - x_c|^2 (r_cell = half side, strict) is taken by
// M2P, phi += sum_m M_m D_m(x - z_c), E -= sum_m M_m D_{m+e_k}(x - z_c); a
// failing leaf by P2P with its particles; a failing inner cell is opened.
//
// One warp walks 32 consecutive targets of the sorted order (neighbours in
// space) together: a shared stack of (cell, lanes) entries, where "lanes" are
// the targets for which the cell is reached (their walks opened its parent).
// Each lane takes its own MAC decision, so every target sees exactly its own
// walk; a cell is visited once for all the lanes that reach it.  The MAC is
// evaluated with explicitly rounded operations (no contraction), in the order
// ((dx dx + dy dy) + dz dz), so the decisions are those of a plain FP64 program.
//
// M2P runs a program built once per (orders, p, outputs, harmonic) on the host:
// the D_k(x - z_c) to compute in graded order, each as at most six terms
// (coefficient, axis of R or none, earlier D) of the recurrence, then the
// contraction with the cell's multipole.  With the harmonic M2L (the handle's
// default) the multipoles are folded onto m_z <= 1 and only the D_k with
// k_z <= 2 are needed: D_{k+2z} = -D_{k+2x} - D_{k+2y} moves every other
// term onto those (the recurrence of such a D_k reads only such D).
#include <cstring>
#include <algorithm>
#include <stdexcept>
#include <vector>

#include "fmm_internal.cuh"
#include "pair.cuh"

namespace fmm {

namespace {

constexpr int kBHMaxWarps = 4;
// pending roots (<= 31) + 7 per level (pop one, push <= 8) over 21 levels + 8
constexpr int kBHStack = 256;

struct BHArgs {
    int64_t n;
    int nsys, nM, nD;
    double theta2;
    const int32_t *nchild, *child, *begin, *end;
    const double *centre, *half;
    const double *px, *py, *pz, *Sm;
    const int32_t *perm;
    const double *M;         // the multipole rows the contraction reads (nM terms per cell)
    const int4 *mt;          // per contraction term: D positions of m, m + e_x, m + e_y, m + e_z
    unsigned long long *count;   // [M2P evaluations, P2P pairs], added per warp
    const int *poff;         // [nD + 1] term ranges of the D program
    const double *pcoef;     // term coefficients
    const int *pw;           // term words: (axis of R + 1) | (position of the D read) << 2
    double *phi_out, *E_out;
};

// D_k(R) = grad^k (1/|R|) for the program's nD entries into D[32 q] (this
// lane's column of its warp's rows), each by the recurrence
// r^2 D_n = -(2 n_i - 1) R_i D_{n-e_i} - (n_i - 1)^2 D_{n-2e_i}
//           - sum_{j != i} [2 n_j R_j D_{n-e_j} + n_j (n_j - 1) D_{n-2e_j}],
// i = the first axis with n_i >= 1, as precomputed terms.
__device__ __forceinline__ void d_program(double R0, double R1, double R2, const BHArgs &a, double *D)
{
    const double r2 = R0 * R0 + R1 * R1 + R2 * R2;
    const double inv_r2 = 1.0 / r2;
    D[0] = rsqrt(r2);
    for (int q = 1; q < a.nD; ++q) {
        const int t0 = __ldg(a.poff + q), t1 = __ldg(a.poff + q + 1);
        double acc = 0.0;
        for (int t = t0; t < t1; ++t) {
            const int w = __ldg(a.pw + t);
            const double c = __ldg(a.pcoef + t);
            const int ax = w & 3;
            const double cr = ax == 0 ? c : c * (ax == 1 ? R0 : (ax == 2 ? R1 : R2));
            acc = fma(cr, D[32 * (w >> 2)], acc);
        }
        D[32 * q] = acc * inv_r2;
    }
}

// SHI > S: every particle carries the orders S..SHI (mixed systems)
template <int S, bool PHI, bool FIELD, int SHI = S>
__global__ void __launch_bounds__(32 * kBHMaxWarps)
k_bh(BHArgs a)
{
    constexpr int nS = Orders<S, SHI>::n;
    constexpr unsigned kAll = 0xffffffffu;
    extern __shared__ double bsm[];
    __shared__ int st_c[kBHMaxWarps][kBHStack];
    __shared__ unsigned st_m[kBHMaxWarps][kBHStack];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *Dl = bsm + (size_t)w * a.nD * 32 + lane;
    const int64_t i = ((int64_t)blockIdx.x * (blockDim.x >> 5) + w) * 32 + lane;
    const bool valid = i < a.n;
    const double x = valid ? a.px[i] : 0.0, y = valid ? a.py[i] : 0.0, z = valid ? a.pz[i] : 0.0;
    double f = 0.0, e0 = 0.0, e1 = 0.0, e2 = 0.0;
    unsigned long long n_m2p = 0, n_p2p = 0;
    int root = 0;
    if (valid) {                          // the last root whose particle range starts at or before i
        int lo = 0, hi = a.nsys - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.begin[mid] <= i) lo = mid; else hi = mid - 1;
        }
        root = lo;
    }
    int top = 0;
    for (unsigned rem = __ballot_sync(kAll, valid); rem;) {
        const int r = __shfl_sync(kAll, root, __ffs(rem) - 1);
        const unsigned m = __ballot_sync(kAll, valid && root == r);
        if (lane == 0) {
            st_c[w][top] = r;
            st_m[w][top] = m;
        }
        ++top;
        rem &= ~m;
    }
    __syncwarp();
    while (top > 0) {
        --top;
        const int c = st_c[w][top];
        const unsigned m = st_m[w][top];
        __syncwarp();                     // read by every lane before a push overwrites it
        bool acc = false;
        double dx = 0.0, dy = 0.0, dz = 0.0;
        if ((m >> lane) & 1u) {
            dx = __dsub_rn(x, a.centre[3 * c]);
            dy = __dsub_rn(y, a.centre[3 * c + 1]);
            dz = __dsub_rn(z, a.centre[3 * c + 2]);
            const double dd = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            const double h = a.half[c];
            acc = __dmul_rn(h, h) < __dmul_rn(a.theta2, dd);
        }
        if (acc) {                        // M2P
            d_program(dx, dy, dz, a, Dl);
            const double *Mc = a.M + (int64_t)c * a.nM;
            double pf = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
            for (int q = 0; q < a.nM; ++q) {
                const double mv = Mc[q];
                const int4 t = a.mt[q];
                if (PHI) pf = fma(mv, Dl[32 * t.x], pf);
                if (FIELD) {
                    g0 = fma(mv, Dl[32 * t.y], g0);
                    g1 = fma(mv, Dl[32 * t.z], g1);
                    g2 = fma(mv, Dl[32 * t.w], g2);
                }
            }
            f += pf;
            e0 -= g0; e1 -= g1; e2 -= g2;
            ++n_m2p;
        }
        const unsigned om = m & ~__ballot_sync(kAll, acc);    // lanes for which c failed
        if (om == 0) continue;
        const int nch = a.nchild[c];
        if (nch == 0) {                   // P2P with the leaf's particles
            const bool mine = (om >> lane) & 1u;
            if (mine) n_p2p += (unsigned long long)(a.end[c] - a.begin[c]);
            for (int j = a.begin[c]; j < a.end[c]; ++j) {
                const double sx = a.px[j], sy = a.py[j], sz = a.pz[j];
                if (mine)
                    pair_orders<S, SHI, PHI, FIELD>(x - sx, y - sy, z - sz, a.Sm + (int64_t)j * nS, f, e0,
                                                    e1, e2);
            }
        } else {                          // open: children pushed last-first, taken in order
            const int ch0 = a.child[c];
            if (lane == 0)
                for (int k = 0; k < nch; ++k) {
                    st_c[w][top + k] = ch0 + nch - 1 - k;
                    st_m[w][top + k] = om;
                }
            top += nch;
            __syncwarp();
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_m2p += __shfl_xor_sync(kAll, n_m2p, o);
        n_p2p += __shfl_xor_sync(kAll, n_p2p, o);
    }
    if (lane == 0) {
        atomicAdd(a.count, n_m2p);
        atomicAdd(a.count + 1, n_p2p);
    }
    if (valid) {
        const int64_t o = a.perm[i];
        if (PHI) a.phi_out[o] = f;
        if (FIELD) {
            a.E_out[3 * o] = e0;
            a.E_out[3 * o + 1] = e1;
            a.E_out[3 * o + 2] = e2;
        }
    }
}

template <int S, int SHI = S>
void launch_bh_s(const BHArgs &a, int want_phi, int want_field, unsigned grid, int threads, size_t smem,
                 cudaStream_t st)
{
    auto go = [&](auto kern) {
        allow_max_dynamic_smem(kern);
        kern<<<grid, threads, smem, st>>>(a);
    };
    if (want_phi && want_field) go(k_bh<S, true, true, SHI>);
    else if (want_phi) go(k_bh<S, true, false, SHI>);
    else go(k_bh<S, false, true, SHI>);
}

// The M2P program (see the file header): D entries, their recurrence terms,
// and per contraction term the D positions of m and m + e_k.
struct BHProgram {
    std::vector<int> off, w;
    std::vector<double> coef;
    std::vector<int4> mt;
};

BHProgram bh_program(int p, bool field, bool harmonic, const std::vector<int> &terms_m)
{
    const MultiIndex &I = multi_index();
    const int P = p + (field ? 1 : 0);
    std::vector<int> at(ntot(P), -1), ks;
    for (int k = 0; k < ntot(P); ++k)
        if (!harmonic || I.nz[k] <= 2) {
            at[k] = (int)ks.size();
            ks.push_back(k);
        }
    BHProgram g;
    g.off.assign(2, 0);                               // D_0 = 1/r: no terms
    for (size_t q = 1; q < ks.size(); ++q) {
        const int k = ks[q];
        const int n[3] = {I.nx[k], I.ny[k], I.nz[k]};
        const int i = n[0] ? 0 : (n[1] ? 1 : 2);
        auto term = [&](double c, int axis, int dax, int dcnt) {
            int m[3] = {n[0], n[1], n[2]};
            m[dax] -= dcnt;
            const int src = at[I(m[0], m[1], m[2])];
            if (src < 0) throw std::logic_error("Barnes-Hut program reads a D it does not compute");
            g.coef.push_back(c);
            g.w.push_back((axis + 1) | src << 2);
        };
        term(-(2.0 * n[i] - 1.0), i, i, 1);
        if (n[i] >= 2) term(-(double)((n[i] - 1) * (n[i] - 1)), -1, i, 2);
        for (int j = 0; j < 3; ++j) {
            if (j == i || n[j] == 0) continue;
            term(-2.0 * n[j], j, j, 1);
            if (n[j] >= 2) term(-(double)(n[j] * (n[j] - 1)), -1, j, 2);
        }
        g.off.push_back((int)g.coef.size());
    }
    for (int m : terms_m) {
        const int x = I.nx[m], y = I.ny[m], z = I.nz[m];
        g.mt.push_back(make_int4(at[m], field ? at[I(x + 1, y, z)] : 0, field ? at[I(x, y + 1, z)] : 0,
                                 field ? at[I(x, y, z + 1)] : 0));
    }
    return g;
}

}  // namespace

fmm_status run_bh(fmm_tree *t, int p, double theta, int want_phi, int want_field, double *phi_out,
                  double *E_out)
{
    cudaStream_t st = t->stream;
    const int s = t->s;
    DevTables tb;
    const int32_t *lut;
    FMM_TRY(upload_tables(t, s, p - s, 0, &tb, &lut));
    FMM_TRY(run_upward(t, tb, false));
    const bool harm = tb.harmonic != 0;
    const double *Mc = (const double *)t->b_M.ptr;
    if (harm) {                                          // multipoles folded onto m_z <= 1
        FMM_TRY(ensure(t, t->b_Mh, 8 * (size_t)t->ncells * tb.nMh));
        launch_fold_m(st, (const double *)t->b_M.ptr, tb.nM, t->ncells, tb, (double *)t->b_Mh.ptr, tb.nMh);
        ++t->launches;
        Mc = (const double *)t->b_Mh.ptr;
    }
    const int key = s | t->s_hi << 2 | p << 4 | (want_field ? 1 : 0) << 9 | (harm ? 1 : 0) << 10;
    if (t->bh_key_s != key) {
        std::vector<int> terms_m;                        // global index of each contraction term
        for (int r = 0; r < tb.nMh; ++r) terms_m.push_back(t->tab.h_rm[r] + tb.m0);
        const BHProgram g = bh_program(p, want_field != 0, harm, terms_m);
        // one buffer: mt (int4) | coef (double) | off | w
        const size_t b_mt = sizeof(int4) * g.mt.size(), b_c = sizeof(double) * g.coef.size();
        const size_t b_off = sizeof(int) * g.off.size(), b_w = sizeof(int) * std::max<size_t>(g.w.size(), 1);
        std::vector<uint8_t> host(b_mt + b_c + b_off + b_w, 0);
        std::memcpy(host.data(), g.mt.data(), b_mt);
        if (b_c) std::memcpy(host.data() + b_mt, g.coef.data(), b_c);
        std::memcpy(host.data() + b_mt + b_c, g.off.data(), b_off);
        if (!g.w.empty()) std::memcpy(host.data() + b_mt + b_c + b_off, g.w.data(), sizeof(int) * g.w.size());
        t->bh_key_s = -1;
        FMM_TRY(ensure(t, t->b_bh_mt, host.size()));
        FMM_TRY(cuda_check(t, cudaMemcpyAsync(t->b_bh_mt.ptr, host.data(), host.size(), cudaMemcpyHostToDevice,
                                              st), "Barnes-Hut program"));
        t->bh_key_s = key;
        t->bh_nD = (int)g.off.size() - 1;
        t->bh_nmt = (int)g.mt.size();
        t->bh_ncoef = (int)g.coef.size();
    }
    FMM_TRY(ensure(t, t->b_bh_cnt, 16));
    FMM_TRY(cuda_check(t, cudaMemsetAsync(t->b_bh_cnt.ptr, 0, 16, st), "memset"));
    BHArgs a;
    a.count = (unsigned long long *)t->b_bh_cnt.ptr;
    a.n = t->n;
    a.nsys = std::max(1, (int)t->sys_off.size() - 1);
    a.nM = t->bh_nmt;
    a.nD = t->bh_nD;
    a.theta2 = theta * theta;
    a.nchild = (const int32_t *)t->b_nchild.ptr;
    a.child = (const int32_t *)t->b_child.ptr;
    a.begin = (const int32_t *)t->b_begin.ptr;
    a.end = (const int32_t *)t->b_end.ptr;
    a.centre = (const double *)t->b_centre.ptr;
    a.half = (const double *)t->b_half.ptr;
    a.px = (const double *)t->b_px.ptr;
    a.py = (const double *)t->b_py.ptr;
    a.pz = (const double *)t->b_pz.ptr;
    a.Sm = (const double *)t->b_S.ptr;
    a.perm = (const int32_t *)t->b_perm.ptr;
    a.M = Mc;
    {
        const uint8_t *base = (const uint8_t *)t->b_bh_mt.ptr;
        const size_t b_mt = sizeof(int4) * t->bh_nmt, b_c = sizeof(double) * t->bh_ncoef;
        a.mt = (const int4 *)base;
        a.pcoef = (const double *)(base + b_mt);
        a.poff = (const int *)(base + b_mt + b_c);
        a.pw = a.poff + (t->bh_nD + 1);
    }
    a.phi_out = phi_out;
    a.E_out = E_out;
    // D rows in shared memory: 32 lanes x nD doubles per warp
    const int wpb = std::max(1, std::min(kBHMaxWarps, (200 * 1024) / (a.nD * 256)));
    const size_t smem = (size_t)wpb * a.nD * 256;
    const unsigned grid = (unsigned)((t->n + 32 * wpb - 1) / (32 * wpb));
    switch (s * 3 + t->s_hi) {
    case 0: launch_bh_s<0>(a, want_phi, want_field, grid, 32 * wpb, smem, st); break;
    case 1: launch_bh_s<0, 1>(a, want_phi, want_field, grid, 32 * wpb, smem, st); break;
    case 2: launch_bh_s<0, 2>(a, want_phi, want_field, grid, 32 * wpb, smem, st); break;
    case 4: launch_bh_s<1>(a, want_phi, want_field, grid, 32 * wpb, smem, st); break;
    case 5: launch_bh_s<1, 2>(a, want_phi, want_field, grid, 32 * wpb, smem, st); break;
    default: launch_bh_s<2>(a, want_phi, want_field, grid, 32 * wpb, smem, st); break;
    }
    ++t->launches;
    t->bh_ran = true;
    return cuda_check(t, cudaGetLastError(), "Barnes-Hut walk");
}

}  // namespace fmm
