// pair.cuh -- the FP64 terms of one source particle seen from one target
// (§2, Eq. (1) with the source moments S of §2):
//   phi_i += sum_{|a|=s} S_{j,a} D_a(R),  E_i -= sum_a S_{j,a} grad D_a(R),  R = x_i - x_j,
// written out per source order (s = 0, 1, 2); r = 0 contributes nothing.
// Shared by the direct sum, the P2P kernels and the Barnes-Hut walk.
#pragma once

namespace fmm {

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

// Moments per particle of the orders SLO..SHI (graded order, shell by shell).
template <int SLO, int SHI>
struct Orders {
    static constexpr int n = ((SHI + 1) * (SHI + 2) * (SHI + 3) - SLO * (SLO + 1) * (SLO + 2)) / 6;
};

// A particle carrying every order SLO..SHI (§2 mixed systems): the sum of the
// pair terms of its shells, the moments of shell s starting after those of
// the lower shells.
template <int SLO, int SHI, bool PHI, bool FIELD>
__device__ __forceinline__ void pair_orders(double dx, double dy, double dz, const double *Sj,
                                            double &f, double &e0, double &e1, double &e2)
{
    pair_fp64<SLO, PHI, FIELD>(dx, dy, dz, Sj, f, e0, e1, e2);
    if constexpr (SHI >= SLO + 1)
        pair_fp64<SLO + 1, PHI, FIELD>(dx, dy, dz, Sj + (SLO + 1) * (SLO + 2) / 2, f, e0, e1, e2);
    if constexpr (SHI >= SLO + 2)
        pair_fp64<SLO + 2, PHI, FIELD>(dx, dy, dz, Sj + (SLO + 1) * (SLO + 2) / 2 + (SLO + 2) * (SLO + 3) / 2,
                                       f, e0, e1, e2);
}

}  // namespace fmm
