/*
 * fmm_oracle.c -- plain, slow, FP64 CPU oracle for the Cartesian-Taylor FMM
 * of Pepper & Fangohr, "fmmgen" (arXiv:2005.12351).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Everything below follows the paper's notation (§2 "Mathematical Basis"):
 *   multi-index n = (nx, ny, nz), n! = nx! ny! nz!, r^n = x^nx y^ny z^nz,
 *   |n| = nx + ny + nz, D_n(R) = grad^n (1/|R|).
 * The kernel is phi = q / |x_b - x_a| (§2, Eq. (1)), with no 4 pi eps0.
 *
 * Readings where the paper is garbled or silent:
 *   - multipole index set  s <= |m| <= p + s, local set |n| <= p, and the
 *     M2L keeps |n| + |m| <= p + s; D_n is needed up to order p + s;
 *   - M2M shift uses (z' - z)^k (new centre minus old), from Eq. (3);
 *   - M2L has no (-1)^n or 1/m! factors (the M2L_1 listing, §3.1);
 *   - L2P sums from |n| = 0 (potential) and from n >= e_k (derivative);
 *   - E = -grad(phi); a source with S_(e_i) = mu_i gives phi = -mu.R/r^3;
 *   - MAC radius r_cell is half the cell side; the MAC is evaluated exactly
 *     in integer units of the finest half-cell (see orc_mac);
 *   - when the MAC fails: two leaves -> P2P, one leaf -> split the other,
 *     else split the larger cell, on a tie split the target; a self pair
 *     (A, A) opens into all ordered child pairs.
 *
 * Compile with -ffp-contract=off: the tree keys and the MAC must be the
 * IEEE results of the written operations.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXORD 16              /* largest |n| any table here supports   */
#define ORC_LEVELS 21              /* key depth: 3 x 21 = 63 key bits        */

/* ------------------------------------------------------------------------ */
/* Multi-index bookkeeping (§3.1: graded lexicographic order               */
/* (000),(100),(010),(001),(200),(110),...).                                */
/* ------------------------------------------------------------------------ */
int orc_ntot(int p) { return p < 0 ? 0 : (p + 1) * (p + 2) * (p + 3) / 6; }

/* Within shell k, nx runs from k down to 0 and, for each nx, ny runs from
 * k - nx down to 0.  a = ny + nz counts how far nx is below k. */
int orc_index(int nx, int ny, int nz)
{
    int k = nx + ny + nz, a = ny + nz;
    return orc_ntot(k - 1) + a * (a + 1) / 2 + nz;
}

static int IX[1000], IY[1000], IZ[1000];   /* ntot(16) = 969 entries */
static int tables_ready = 0;

static void make_tables(void)
{
    if (tables_ready) return;
    int idx = 0;
    for (int k = 0; k <= ORC_MAXORD; ++k)
        for (int nx = k; nx >= 0; --nx)
            for (int ny = k - nx; ny >= 0; --ny) {
                IX[idx] = nx; IY[idx] = ny; IZ[idx] = k - nx - ny; ++idx;
            }
    tables_ready = 1;
}

void orc_multi_index(int idx, int *nx, int *ny, int *nz)
{
    make_tables();
    *nx = IX[idx]; *ny = IY[idx]; *nz = IZ[idx];
}

/* r^k / k! for a 3-vector d, computed directly (§2 notation). */
static double mono(const double d[3], int kx, int ky, int kz)
{
    double t = 1.0;
    for (int i = 1; i <= kx; ++i) t *= d[0] / i;
    for (int i = 1; i <= ky; ++i) t *= d[1] / i;
    for (int i = 1; i <= kz; ++i) t *= d[2] / i;
    return t;
}

/* ------------------------------------------------------------------------ */
/* Derivative tensors D_n(R) = grad^n (1/r), |n| <= order (§3.1, the        */
/* derivatives of 1/r used by M2L; recurrence in the spirit of Challacombe  */
/* et al. cited there).                                                      */
/*                                                                           */
/* From r^2 d_i(1/r) = -R_i (1/r), Leibniz' rule applied with d^m gives, for */
/* n = m + e_i:                                                              */
/*  r^2 D_n = -R_i D_m - m_i D_{m-e_i}                                       */
/*            - 2 sum_j m_j R_j D_{m+e_i-e_j} - sum_j m_j (m_j-1) D_{m+e_i-2e_j} */
/* Here i is the axis of the largest component of n (lowest axis on ties).   */
/* ------------------------------------------------------------------------ */
void orc_derivatives(double x, double y, double z, int order, double *D)
{
    make_tables();
    double R[3] = {x, y, z};
    double r2 = x * x + y * y + z * z;
    D[0] = 1.0 / sqrt(r2);
    for (int idx = 1; idx < orc_ntot(order); ++idx) {
        int n[3] = {IX[idx], IY[idx], IZ[idx]};
        int i = 0;
        if (n[1] > n[i]) i = 1;
        if (n[2] > n[i]) i = 2;
        int m[3] = {n[0], n[1], n[2]};
        m[i] -= 1;
        double acc = -R[i] * D[orc_index(m[0], m[1], m[2])];
        if (m[i] >= 1) {
            int t[3] = {m[0], m[1], m[2]};
            t[i] -= 1;
            acc -= m[i] * D[orc_index(t[0], t[1], t[2])];
        }
        for (int j = 0; j < 3; ++j) {
            if (m[j] >= 1) {
                int t[3] = {m[0], m[1], m[2]};
                t[i] += 1; t[j] -= 1;
                acc -= 2.0 * m[j] * R[j] * D[orc_index(t[0], t[1], t[2])];
            }
            if (m[j] >= 2) {
                int t[3] = {m[0], m[1], m[2]};
                t[i] += 1; t[j] -= 2;
                acc -= (double)m[j] * (m[j] - 1) * D[orc_index(t[0], t[1], t[2])];
            }
        }
        D[idx] = acc / r2;
    }
}

/* ------------------------------------------------------------------------ */
/* Operators on single cells.  Storage: M over s <= |m| <= p+s at offset     */
/* index(m) - ntot(s-1); L over |n| <= p at offset index(n); source moments   */
/* S_j over |a| = s at offset index(a) - ntot(s-1).                           */
/* ------------------------------------------------------------------------ */
int orc_n_multipole(int s, int p) { return orc_ntot(p + s) - orc_ntot(s - 1); }
int orc_n_local(int p) { return orc_ntot(p); }

/* Source moments of a system whose particles carry the orders s_lo..s_hi
 * (§2: "mixed systems"): the graded indices ntot(s_lo - 1) .. ntot(s_hi) - 1,
 * S_{j,a} in that order per particle.  A single order s is s_lo = s_hi = s. */
static int n_src(int s_lo, int s_hi) { return orc_ntot(s_hi) - orc_ntot(s_lo - 1); }

/* P2M, §2 Eq. (5) with Eq. (3)'s sign: M_m(z) = sum_j sum_{a<=m, s_lo<=|a|<=s_hi}
 * (z - x_j)^(m-a)/(m-a)! S_{j,a}, for s_lo <= |m| <= p + s_lo. */
void orc_p2m_orders(int s_lo, int s_hi, int p, const double zc[3], int64_t cnt, const double *pos,
                    const double *S, double *M)
{
    make_tables();
    int s = s_lo;
    int m0 = orc_ntot(s - 1), nM = orc_n_multipole(s, p), nS = n_src(s_lo, s_hi);
    for (int64_t j = 0; j < cnt; ++j) {
        double d[3] = {zc[0] - pos[3 * j], zc[1] - pos[3 * j + 1], zc[2] - pos[3 * j + 2]};
        for (int mi = 0; mi < nM; ++mi) {
            int idx = mi + m0;
            for (int ai = 0; ai < nS; ++ai) {
                int a = ai + m0;
                int kx = IX[idx] - IX[a], ky = IY[idx] - IY[a], kz = IZ[idx] - IZ[a];
                if (kx < 0 || ky < 0 || kz < 0) continue;
                M[mi] += mono(d, kx, ky, kz) * S[nS * j + ai];
            }
        }
    }
}

void orc_p2m(int s, int p, const double zc[3], int64_t cnt, const double *pos, const double *S,
             double *M)
{
    orc_p2m_orders(s, s, p, zc, cnt, pos, S, M);
}

/* M2M, §2 Eq. (4) with the sign fixed by Eq. (3):
 * M_n(zp) += sum_{k<=n, |n-k|>=s} (zp - zc)^k/k! M_{n-k}(zc). */
void orc_m2m(int s, int p, const double zc[3], const double zp[3], const double *Mc, double *Mp)
{
    make_tables();
    int m0 = orc_ntot(s - 1), nM = orc_n_multipole(s, p);
    double d[3] = {zp[0] - zc[0], zp[1] - zc[1], zp[2] - zc[2]};
    for (int ni = 0; ni < nM; ++ni) {
        int n = ni + m0;
        double acc = 0.0;
        for (int qi = 0; qi < nM; ++qi) {          /* q = n - k must lie in the M set */
            int q = qi + m0;
            int kx = IX[n] - IX[q], ky = IY[n] - IY[q], kz = IZ[n] - IZ[q];
            if (kx < 0 || ky < 0 || kz < 0) continue;
            acc += mono(d, kx, ky, kz) * Mc[qi];
        }
        Mp[ni] += acc;
    }
}

/* M2L, §2 Eq. (8) read through the M2L_1 listing (§3.1):
 * L_n(zt) += sum_{m, |n|+|m|<=p+s} D_{n+m}(zt - zs) M_m(zs). */
void orc_m2l(int s, int p, const double zt[3], const double zs[3], const double *Ms, double *Lt)
{
    make_tables();
    double D[1000];
    orc_derivatives(zt[0] - zs[0], zt[1] - zs[1], zt[2] - zs[2], p + s, D);
    int m0 = orc_ntot(s - 1), nM = orc_n_multipole(s, p), nL = orc_n_local(p);
    for (int n = 0; n < nL; ++n) {
        double acc = 0.0;
        for (int mi = 0; mi < nM; ++mi) {
            int m = mi + m0;
            int nm = IX[n] + IY[n] + IZ[n] + IX[m] + IY[m] + IZ[m];
            if (nm > p + s) continue;
            acc += D[orc_index(IX[n] + IX[m], IY[n] + IY[m], IZ[n] + IZ[m])] * Ms[mi];
        }
        Lt[n] += acc;
    }
}

/* L2L (named in §3.1, no formula printed): Taylor shift of the local
 * expansion, L_n(zc) += sum_{k, |n+k|<=p} (zc - zp)^k/k! L_{n+k}(zp). */
void orc_l2l(int p, const double zp[3], const double zc[3], const double *Lp, double *Lc)
{
    make_tables();
    int nL = orc_n_local(p);
    double d[3] = {zc[0] - zp[0], zc[1] - zp[1], zc[2] - zp[2]};
    for (int n = 0; n < nL; ++n) {
        double acc = 0.0;
        for (int q = 0; q < nL; ++q) {            /* q = n + k */
            int kx = IX[q] - IX[n], ky = IY[q] - IY[n], kz = IZ[q] - IZ[n];
            if (kx < 0 || ky < 0 || kz < 0) continue;
            acc += mono(d, kx, ky, kz) * Lp[q];
        }
        Lc[n] += acc;
    }
}

/* L2P, §2 Eqs. (9) and (10) with lower limits 0 and e_k:
 * phi = sum_n (x-z)^n/n! L_n, d_k phi = sum_{n>=e_k} (x-z)^(n-e_k)/(n-e_k)! L_n. */
void orc_l2p(int p, const double z[3], const double *L, const double x[3], double *phi, double grad[3])
{
    make_tables();
    double d[3] = {x[0] - z[0], x[1] - z[1], x[2] - z[2]};
    double f = 0.0, g[3] = {0.0, 0.0, 0.0};
    for (int n = 0; n < orc_n_local(p); ++n) {
        f += mono(d, IX[n], IY[n], IZ[n]) * L[n];
        if (IX[n] >= 1) g[0] += mono(d, IX[n] - 1, IY[n], IZ[n]) * L[n];
        if (IY[n] >= 1) g[1] += mono(d, IX[n], IY[n] - 1, IZ[n]) * L[n];
        if (IZ[n] >= 1) g[2] += mono(d, IX[n], IY[n], IZ[n] - 1) * L[n];
    }
    *phi = f; grad[0] = g[0]; grad[1] = g[1]; grad[2] = g[2];
}

/* One source j seen at target x (P2P, §3.1): phi = sum_{|a|=s} S_a D_a(x - x_j),
 * d_k phi = sum_a S_a D_{a+e_k}(x - x_j).  A coincident pair contributes 0. */
void orc_p2p_pair_orders(int s_lo, int s_hi, const double xt[3], const double xs[3], const double *S,
                         double *phi, double grad[3])
{
    make_tables();
    double R[3] = {xt[0] - xs[0], xt[1] - xs[1], xt[2] - xs[2]};
    *phi = 0.0; grad[0] = grad[1] = grad[2] = 0.0;
    if (R[0] == 0.0 && R[1] == 0.0 && R[2] == 0.0) return;
    double D[64];
    orc_derivatives(R[0], R[1], R[2], s_hi + 1, D);
    int m0 = orc_ntot(s_lo - 1), nS = n_src(s_lo, s_hi);
    for (int ai = 0; ai < nS; ++ai) {
        int a = ai + m0;
        *phi += S[ai] * D[a];
        grad[0] += S[ai] * D[orc_index(IX[a] + 1, IY[a], IZ[a])];
        grad[1] += S[ai] * D[orc_index(IX[a], IY[a] + 1, IZ[a])];
        grad[2] += S[ai] * D[orc_index(IX[a], IY[a], IZ[a] + 1)];
    }
}

void orc_p2p_pair(int s, const double xt[3], const double xs[3], const double *S, double *phi,
                  double grad[3])
{
    orc_p2p_pair_orders(s, s, xt, xs, S, phi, grad);
}

/* ------------------------------------------------------------------------ */
/* Direct sum: the plain definition the FMM approximates.                   */
/* phi_i = sum_{j != i} sum_{|a|=s} S_{j,a} D_a(x_i - x_j), E_i = -grad phi_i, */
/* accumulated with Neumaier's compensated summation.                        */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } nsum;
static void nadd(nsum *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}

void orc_direct_orders(int s_lo, int s_hi, int64_t n, const double *pos, const double *S,
                       int64_t ntarget, const int64_t *targets, double *phi, double *E)
{
    make_tables();
    int nS = n_src(s_lo, s_hi);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < ntarget; ++t) {
        int64_t i = targets ? targets[t] : t;
        nsum f = {0, 0}, g0 = {0, 0}, g1 = {0, 0}, g2 = {0, 0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double pf, pg[3];
            orc_p2p_pair_orders(s_lo, s_hi, pos + 3 * i, pos + 3 * j, S + nS * j, &pf, pg);
            nadd(&f, pf); nadd(&g0, pg[0]); nadd(&g1, pg[1]); nadd(&g2, pg[2]);
        }
        phi[t] = f.s + f.c;
        E[3 * t] = -(g0.s + g0.c);
        E[3 * t + 1] = -(g1.s + g1.c);
        E[3 * t + 2] = -(g2.s + g2.c);
    }
}

void orc_direct(int s, int64_t n, const double *pos, const double *S, int64_t ntarget,
                const int64_t *targets, double *phi, double *E)
{
    orc_direct_orders(s, s, n, pos, S, ntarget, targets, phi, E);
}

/* ------------------------------------------------------------------------ */
/* Octree (§3.2: split an octant while it holds more than n_crit particles; */
/* the expansion centre is the geometric cell centre).                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    int ncrit;
    double lo[3], side;
    uint64_t *key;          /* Morton key per ORIGINAL particle            */
    int64_t *perm;          /* perm[k] = original index of sorted slot k    */
    int64_t ncells;
    int nlevels;            /* 1 + deepest level                            */
    int *level;
    int64_t *ci;            /* integer cell coordinates, 3 per cell         */
    int64_t *begin, *end;   /* sorted-particle range                        */
    int64_t *parent, *child_first;
    int *nchild;
    double *centre, *halfw; /* 3 per cell, 1 per cell                       */
    int64_t *level_begin;   /* cells of level l are [level_begin[l], level_begin[l+1]) */
    /* interaction lists, sorted by (target, source) */
    double theta;
    int64_t nm2l, np2p;
    int64_t *m2l, *p2p;     /* pairs (target, source), 2 per pair           */
} orc_tree;

/* Root box: lo = per-axis minimum; side = smallest power of two >= the
 * largest per-axis extent (1 when all points coincide).  Integer coords
 * q = min(floor((x - lo) * 2^21 / side), 2^21 - 1); the scale is a power of
 * two, so only x - lo rounds. */
static uint64_t morton(uint64_t qx, uint64_t qy, uint64_t qz)
{
    uint64_t k = 0;
    for (int b = 0; b < ORC_LEVELS; ++b) {
        k |= ((qx >> b) & 1u) << (3 * b + 2);
        k |= ((qy >> b) & 1u) << (3 * b + 1);
        k |= ((qz >> b) & 1u) << (3 * b);
    }
    return k;
}

static const uint64_t *g_sort_keys;
static int cmp_key_then_index(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    if (g_sort_keys[i] < g_sort_keys[j]) return -1;
    if (g_sort_keys[i] > g_sort_keys[j]) return 1;
    return (i > j) - (i < j);
}

static int child_digit(uint64_t key, int child_level)
{
    return (int)((key >> (3 * (ORC_LEVELS - child_level))) & 7u);
}

orc_tree *orc_tree_build(int64_t n, const double *pos, int ncrit)
{
    orc_tree *t = (orc_tree *)calloc(1, sizeof(orc_tree));
    t->n = n; t->ncrit = ncrit;
    t->key = (uint64_t *)malloc(sizeof(uint64_t) * (n > 0 ? n : 1));
    t->perm = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    if (n == 0) { t->side = 1.0; return t; }

    double hi[3];
    for (int d = 0; d < 3; ++d) { t->lo[d] = pos[d]; hi[d] = pos[d]; }
    for (int64_t i = 1; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            if (pos[3 * i + d] < t->lo[d]) t->lo[d] = pos[3 * i + d];
            if (pos[3 * i + d] > hi[d]) hi[d] = pos[3 * i + d];
        }
    double ext = 0.0;
    for (int d = 0; d < 3; ++d) if (hi[d] - t->lo[d] > ext) ext = hi[d] - t->lo[d];
    double side = 1.0;
    if (ext > 0.0) {
        while (side < ext) side *= 2.0;
        while (side / 2.0 >= ext) side /= 2.0;
    }
    t->side = side;
    double scale = ldexp(1.0, ORC_LEVELS) / side;
    const uint64_t qmax = (1u << ORC_LEVELS) - 1;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t q[3];
        for (int d = 0; d < 3; ++d) {
            double u = floor((pos[3 * i + d] - t->lo[d]) * scale);
            q[d] = (uint64_t)u;
            if (q[d] > qmax) q[d] = qmax;
        }
        t->key[i] = morton(q[0], q[1], q[2]);
        t->perm[i] = i;
    }
    g_sort_keys = t->key;
    qsort(t->perm, (size_t)n, sizeof(int64_t), cmp_key_then_index);

    /* breadth-first cell construction */
    int64_t cap = 1024, nc = 1;
    t->level = malloc(sizeof(int) * cap);       t->ci = malloc(sizeof(int64_t) * 3 * cap);
    t->begin = malloc(sizeof(int64_t) * cap);   t->end = malloc(sizeof(int64_t) * cap);
    t->parent = malloc(sizeof(int64_t) * cap);  t->child_first = malloc(sizeof(int64_t) * cap);
    t->nchild = malloc(sizeof(int) * cap);
    t->level[0] = 0; t->ci[0] = t->ci[1] = t->ci[2] = 0;
    t->begin[0] = 0; t->end[0] = n; t->parent[0] = -1;
    for (int64_t c = 0; c < nc; ++c) {
        t->child_first[c] = -1; t->nchild[c] = 0;
        int64_t cnt = t->end[c] - t->begin[c];
        if (!(cnt > ncrit && t->level[c] < ORC_LEVELS)) continue;
        int cl = t->level[c] + 1;
        int64_t k = t->begin[c];
        for (int o = 0; o < 8; ++o) {
            int64_t b = k;
            while (k < t->end[c] && child_digit(t->key[t->perm[k]], cl) == o) ++k;
            if (k == b) continue;
            if (nc == cap) {
                cap *= 2;
                t->level = realloc(t->level, sizeof(int) * cap);
                t->ci = realloc(t->ci, sizeof(int64_t) * 3 * cap);
                t->begin = realloc(t->begin, sizeof(int64_t) * cap);
                t->end = realloc(t->end, sizeof(int64_t) * cap);
                t->parent = realloc(t->parent, sizeof(int64_t) * cap);
                t->child_first = realloc(t->child_first, sizeof(int64_t) * cap);
                t->nchild = realloc(t->nchild, sizeof(int) * cap);
            }
            if (t->nchild[c] == 0) t->child_first[c] = nc;
            t->nchild[c] += 1;
            t->level[nc] = cl;
            t->ci[3 * nc] = 2 * t->ci[3 * c] + ((o >> 2) & 1);
            t->ci[3 * nc + 1] = 2 * t->ci[3 * c + 1] + ((o >> 1) & 1);
            t->ci[3 * nc + 2] = 2 * t->ci[3 * c + 2] + (o & 1);
            t->begin[nc] = b; t->end[nc] = k; t->parent[nc] = c;
            ++nc;
        }
    }
    t->ncells = nc;
    t->centre = malloc(sizeof(double) * 3 * nc);
    t->halfw = malloc(sizeof(double) * nc);
    t->nlevels = t->level[nc - 1] + 1;
    t->level_begin = malloc(sizeof(int64_t) * (t->nlevels + 1));
    for (int l = 0; l <= t->nlevels; ++l) t->level_begin[l] = nc;
    for (int64_t c = nc - 1; c >= 0; --c) t->level_begin[t->level[c]] = c;
    for (int64_t c = 0; c < nc; ++c) {
        double h = ldexp(side, -(t->level[c] + 1));          /* half the side */
        t->halfw[c] = h;
        for (int d = 0; d < 3; ++d)
            t->centre[3 * c + d] = t->lo[d] + (double)(2 * t->ci[3 * c + d] + 1) * h;
    }
    return t;
}

/* MAC, §3.2 Eq. (13): (r_A + r_B) / R < theta with r = half the side.
 * Centres and radii are integers in units of the finest half-cell
 * u = side / 2^22 (centre = (2c+1) 2^(21-l) u, radius = 2^(21-l) u), so the
 * test (r_A + r_B)^2 < (theta*theta) * |dc|^2 has exact integer operands;
 * only the product on the right rounds, once. */
static int orc_mac(const orc_tree *t, int64_t a, int64_t b, double theta)
{
    int64_t ra = (int64_t)1 << (ORC_LEVELS - t->level[a]);
    int64_t rb = (int64_t)1 << (ORC_LEVELS - t->level[b]);
    int64_t d2 = 0;
    for (int d = 0; d < 3; ++d) {
        int64_t ca = (2 * t->ci[3 * a + d] + 1) * ra;
        int64_t cb = (2 * t->ci[3 * b + d] + 1) * rb;
        d2 += (ca - cb) * (ca - cb);
    }
    double lhs = (double)((ra + rb) * (ra + rb));
    double rhs = (theta * theta) * (double)d2;
    return lhs < rhs;
}

typedef struct { int64_t *v; int64_t n, cap; } pairvec;
static void push_pair(pairvec *p, int64_t a, int64_t b)
{
    if (p->n == p->cap) {
        p->cap = p->cap ? 2 * p->cap : 1024;
        p->v = realloc(p->v, sizeof(int64_t) * 2 * p->cap);
    }
    p->v[2 * p->n] = a; p->v[2 * p->n + 1] = b; ++p->n;
}

/* Dual-tree traversal (§3.2): accepted pairs interact by M2L, leaf pairs
 * that fail interact directly; the lists are stored once and sorted. */
static void traverse(const orc_tree *t, int64_t a, int64_t b, double theta,
                     pairvec *m2l, pairvec *p2p)
{
    int leaf_a = t->nchild[a] == 0, leaf_b = t->nchild[b] == 0;
    if (a == b) {
        if (leaf_a) { push_pair(p2p, a, a); return; }
        for (int i = 0; i < t->nchild[a]; ++i)
            for (int j = 0; j < t->nchild[a]; ++j)
                traverse(t, t->child_first[a] + i, t->child_first[a] + j, theta, m2l, p2p);
        return;
    }
    if (orc_mac(t, a, b, theta)) { push_pair(m2l, a, b); return; }
    if (leaf_a && leaf_b) { push_pair(p2p, a, b); return; }
    int split_a;
    if (leaf_a) split_a = 0;
    else if (leaf_b) split_a = 1;
    else split_a = t->level[a] <= t->level[b];   /* larger (or equal): target */
    if (split_a) {
        for (int i = 0; i < t->nchild[a]; ++i)
            traverse(t, t->child_first[a] + i, b, theta, m2l, p2p);
    } else {
        for (int j = 0; j < t->nchild[b]; ++j)
            traverse(t, a, t->child_first[b] + j, theta, m2l, p2p);
    }
}

static int cmp_pair(const void *x, const void *y)
{
    const int64_t *a = (const int64_t *)x, *b = (const int64_t *)y;
    if (a[0] != b[0]) return (a[0] > b[0]) - (a[0] < b[0]);
    return (a[1] > b[1]) - (a[1] < b[1]);
}

void orc_tree_lists(orc_tree *t, double theta)
{
    free(t->m2l); free(t->p2p);
    t->m2l = t->p2p = NULL; t->nm2l = t->np2p = 0; t->theta = theta;
    if (t->n == 0) return;
    pairvec m2l = {0}, p2p = {0};
    traverse(t, 0, 0, theta, &m2l, &p2p);
    if (m2l.n) qsort(m2l.v, (size_t)m2l.n, 2 * sizeof(int64_t), cmp_pair);
    if (p2p.n) qsort(p2p.v, (size_t)p2p.n, 2 * sizeof(int64_t), cmp_pair);
    t->m2l = m2l.v; t->nm2l = m2l.n;
    t->p2p = p2p.v; t->np2p = p2p.n;
}

void orc_tree_free(orc_tree *t)
{
    if (!t) return;
    free(t->key); free(t->perm); free(t->level); free(t->ci); free(t->begin);
    free(t->end); free(t->parent); free(t->child_first); free(t->nchild);
    free(t->centre); free(t->halfw); free(t->level_begin); free(t->m2l); free(t->p2p);
    free(t);
}

/* accessors (plain copies into caller buffers) */
void orc_tree_sizes(const orc_tree *t, int64_t *out)
{
    out[0] = t->n; out[1] = t->ncells; out[2] = t->nlevels;
    out[3] = t->nm2l; out[4] = t->np2p;
}
void orc_tree_box(const orc_tree *t, double *out)
{
    out[0] = t->lo[0]; out[1] = t->lo[1]; out[2] = t->lo[2]; out[3] = t->side;
}
void orc_tree_particles(const orc_tree *t, uint64_t *key_sorted, int64_t *perm)
{
    for (int64_t k = 0; k < t->n; ++k) {
        perm[k] = t->perm[k];
        key_sorted[k] = t->key[t->perm[k]];
    }
}
void orc_tree_cells(const orc_tree *t, int32_t *level, int64_t *ci, int64_t *begin, int64_t *end,
                    int64_t *parent, int64_t *child_first, int32_t *nchild,
                    double *centre, double *halfw)
{
    for (int64_t c = 0; c < t->ncells; ++c) {
        level[c] = t->level[c];
        for (int d = 0; d < 3; ++d) { ci[3 * c + d] = t->ci[3 * c + d]; centre[3 * c + d] = t->centre[3 * c + d]; }
        begin[c] = t->begin[c]; end[c] = t->end[c]; parent[c] = t->parent[c];
        child_first[c] = t->child_first[c]; nchild[c] = t->nchild[c]; halfw[c] = t->halfw[c];
    }
}
void orc_tree_get_lists(const orc_tree *t, int64_t *m2l, int64_t *p2p)
{
    memcpy(m2l, t->m2l, sizeof(int64_t) * 2 * t->nm2l);
    memcpy(p2p, t->p2p, sizeof(int64_t) * 2 * t->np2p);
}

/* ------------------------------------------------------------------------ */
/* Scalar FMM on the tree (§3.2): P2M at leaves, M2M upward, M2L over the   */
/* stored lists, L2L downward, L2P + P2P at the leaves.                      */
/* If targets != NULL, only those particles (original indices) are output;  */
/* the downward pass then runs only on their leaves' ancestor chains.        */
/* ------------------------------------------------------------------------ */
int orc_fmm_orders(const orc_tree *t, const double *pos_orig, int s_lo, int s_hi, int p,
                   const double *S_orig, int64_t ntarget, const int64_t *targets, double *phi,
                   double *E)
{
    make_tables();
    int s = s_lo;
    if (p + s + 1 > ORC_MAXORD || p < 0 || s < 0 || s_hi < s_lo || s_hi > 2) return -1;
    int64_t n = t->n, nc = t->ncells;
    if (n == 0 || ntarget == 0) return 0;
    int nM = orc_n_multipole(s, p), nL = orc_n_local(p), nS = n_src(s_lo, s_hi);

    double *pos = malloc(sizeof(double) * 3 * n), *S = malloc(sizeof(double) * nS * n);
    for (int64_t k = 0; k < n; ++k) {
        int64_t o = t->perm[k];
        for (int d = 0; d < 3; ++d) pos[3 * k + d] = pos_orig[3 * o + d];
        for (int a = 0; a < nS; ++a) S[nS * k + a] = S_orig[nS * o + a];
    }
    int64_t *leaf_of = malloc(sizeof(int64_t) * n);          /* sorted slot -> leaf */
    for (int64_t c = 0; c < nc; ++c)
        if (t->nchild[c] == 0)
            for (int64_t k = t->begin[c]; k < t->end[c]; ++k) leaf_of[k] = c;

    /* upward pass */
    double *M = calloc((size_t)nc * nM, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < nc; ++c)
        if (t->nchild[c] == 0)
            orc_p2m_orders(s_lo, s_hi, p, t->centre + 3 * c, t->end[c] - t->begin[c],
                           pos + 3 * t->begin[c], S + nS * t->begin[c], M + (size_t)nM * c);
    for (int l = t->nlevels - 2; l >= 0; --l) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t c = t->level_begin[l]; c < t->level_begin[l + 1]; ++c)
            for (int i = 0; i < t->nchild[c]; ++i) {
                int64_t ch = t->child_first[c] + i;
                orc_m2m(s, p, t->centre + 3 * ch, t->centre + 3 * c, M + (size_t)nM * ch,
                        M + (size_t)nM * c);
            }
    }

    /* which cells need a local expansion: every cell, or the ancestors of
     * the requested targets' leaves */
    char *need = calloc((size_t)nc, 1);
    int64_t *rank = malloc(sizeof(int64_t) * n);       /* rank[original] = sorted slot */
    for (int64_t k = 0; k < n; ++k) rank[t->perm[k]] = k;
    int64_t *tslot = malloc(sizeof(int64_t) * ntarget);
    for (int64_t q = 0; q < ntarget; ++q) tslot[q] = rank[targets ? targets[q] : q];
    if (!targets) { memset(need, 1, (size_t)nc); }
    else {
        for (int64_t q = 0; q < ntarget; ++q)
            for (int64_t c = leaf_of[tslot[q]]; c >= 0; c = t->parent[c]) need[c] = 1;
    }

    /* M2L over the stored (target-sorted) list */
    int64_t *m2l_first = malloc(sizeof(int64_t) * (nc + 1));
    {
        int64_t k = 0;
        for (int64_t c = 0; c <= nc; ++c) {
            while (k < t->nm2l && t->m2l[2 * k] < c) ++k;
            m2l_first[c] = k;
        }
    }
    double *L = calloc((size_t)nc * nL, sizeof(double));
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t c = 0; c < nc; ++c) {
        if (!need[c]) continue;
        for (int64_t k = m2l_first[c]; k < m2l_first[c + 1]; ++k) {
            int64_t b = t->m2l[2 * k + 1];
            orc_m2l(s, p, t->centre + 3 * c, t->centre + 3 * b, M + (size_t)nM * b, L + (size_t)nL * c);
        }
    }
    /* L2L, level by level downward */
    for (int l = 1; l < t->nlevels; ++l) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t c = t->level_begin[l]; c < t->level_begin[l + 1]; ++c) {
            if (!need[c]) continue;
            int64_t pa = t->parent[c];
            orc_l2l(p, t->centre + 3 * pa, t->centre + 3 * c, L + (size_t)nL * pa, L + (size_t)nL * c);
        }
    }
    /* P2P list by target leaf */
    int64_t *p2p_first = malloc(sizeof(int64_t) * (nc + 1));
    {
        int64_t k = 0;
        for (int64_t c = 0; c <= nc; ++c) {
            while (k < t->np2p && t->p2p[2 * k] < c) ++k;
            p2p_first[c] = k;
        }
    }
    /* L2P + P2P per target particle */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < ntarget; ++q) {
        int64_t k = tslot[q], c = leaf_of[k];
        double f, g[3];
        orc_l2p(p, t->centre + 3 * c, L + (size_t)nL * c, pos + 3 * k, &f, g);
        for (int64_t e = p2p_first[c]; e < p2p_first[c + 1]; ++e) {
            int64_t b = t->p2p[2 * e + 1];
            for (int64_t j = t->begin[b]; j < t->end[b]; ++j) {
                if (j == k) continue;
                double pf, pg[3];
                orc_p2p_pair_orders(s_lo, s_hi, pos + 3 * k, pos + 3 * j, S + nS * j, &pf, pg);
                f += pf; g[0] += pg[0]; g[1] += pg[1]; g[2] += pg[2];
            }
        }
        phi[q] = f;
        E[3 * q] = -g[0]; E[3 * q + 1] = -g[1]; E[3 * q + 2] = -g[2];
    }
    free(pos); free(S); free(leaf_of); free(M); free(need); free(rank); free(tslot);
    free(m2l_first); free(L); free(p2p_first);
    return 0;
}

int orc_fmm(const orc_tree *t, const double *pos_orig, int s, int p, const double *S_orig,
            int64_t ntarget, const int64_t *targets, double *phi, double *E)
{
    return orc_fmm_orders(t, pos_orig, s, s, p, S_orig, ntarget, targets, phi, E);
}

/* ------------------------------------------------------------------------ */
/* Multipolar Barnes-Hut (§2 multipole potential; §3.2 Methods).             */
/* M2P: phi(x) = sum_{s <= |m| <= p} M_m D_m(x - z) and grad phi(x) =         */
/* sum M_m D_{m + e_k}(x - z): the multipole sum of order p that the paper's  */
/* BH formula runs over (|n| from s to p), differentiated exactly.  The       */
/* multipoles s <= |m| <= p are those of the FMM storage at order p - s.      */
/* ------------------------------------------------------------------------ */
void orc_m2p(int s, int p, const double z[3], const double *M, const double x[3], double *phi,
             double grad[3])
{
    make_tables();
    double R[3] = {x[0] - z[0], x[1] - z[1], x[2] - z[2]};
    int m0 = orc_ntot(s - 1), nM = orc_ntot(p) - m0;
    double *D = malloc(sizeof(double) * orc_ntot(p + 1));
    orc_derivatives(R[0], R[1], R[2], p + 1, D);
    *phi = 0.0; grad[0] = grad[1] = grad[2] = 0.0;
    for (int mi = 0; mi < nM; ++mi) {
        int m = mi + m0;
        *phi += M[mi] * D[m];
        grad[0] += M[mi] * D[orc_index(IX[m] + 1, IY[m], IZ[m])];
        grad[1] += M[mi] * D[orc_index(IX[m], IY[m] + 1, IZ[m])];
        grad[2] += M[mi] * D[orc_index(IX[m], IY[m], IZ[m] + 1)];
    }
    free(D);
}

typedef struct {
    const orc_tree *t;
    const double *pos, *S, *M;
    int s, s_hi, p, nM, nS;
    double theta2;
} bh_ctx;

/* The walk of one target from cell c down (§3.2): a cell with
 * r_cell^2 < theta^2 |x - x_c|^2 (r_cell = half side, strict) is taken by
 * M2P; otherwise a leaf by P2P with its particles (the target itself and
 * coincident points excluded), otherwise its children in order. */
static void bh_walk(const bh_ctx *b, int64_t c, int64_t self, const double x[3], double *f,
                    double g[3])
{
    const orc_tree *t = b->t;
    const double *zc = t->centre + 3 * c;
    double d0 = x[0] - zc[0], d1 = x[1] - zc[1], d2 = x[2] - zc[2];
    double dd = d0 * d0 + d1 * d1 + d2 * d2;
    double h = t->halfw[c];
    if (h * h < b->theta2 * dd) {
        double pf, pg[3];
        orc_m2p(b->s, b->p, zc, b->M + (size_t)b->nM * c, x, &pf, pg);
        *f += pf; g[0] += pg[0]; g[1] += pg[1]; g[2] += pg[2];
        return;
    }
    if (t->nchild[c] == 0) {
        for (int64_t j = t->begin[c]; j < t->end[c]; ++j) {
            if (j == self) continue;
            double pf, pg[3];
            orc_p2p_pair_orders(b->s, b->s_hi, x, b->pos + 3 * j, b->S + (size_t)b->nS * j, &pf, pg);
            *f += pf; g[0] += pg[0]; g[1] += pg[1]; g[2] += pg[2];
        }
        return;
    }
    for (int i = 0; i < t->nchild[c]; ++i) bh_walk(b, t->child_first[c] + i, self, x, f, g);
}

/* Barnes-Hut on the tree: P2M at the leaves and M2M upward (order p - s,
 * i.e. s <= |m| <= p), then one walk from the root per requested target. */
int orc_bh_orders(const orc_tree *t, const double *pos_orig, int s_lo, int s_hi, int p,
                  const double *S_orig, double theta, int64_t ntarget, const int64_t *targets,
                  double *phi, double *E)
{
    make_tables();
    int s = s_lo;
    if (s < 0 || s_hi < s_lo || s_hi > 2 || p < s || p + 1 > ORC_MAXORD || !(theta >= 0.0)) return -1;
    int64_t n = t->n, nc = t->ncells;
    if (n == 0 || ntarget == 0) return 0;
    int pt = p - s, nM = orc_n_multipole(s, pt), nS = n_src(s_lo, s_hi);
    double *pos = malloc(sizeof(double) * 3 * n), *S = malloc(sizeof(double) * nS * n);
    for (int64_t k = 0; k < n; ++k) {
        int64_t o = t->perm[k];
        for (int d = 0; d < 3; ++d) pos[3 * k + d] = pos_orig[3 * o + d];
        for (int a = 0; a < nS; ++a) S[nS * k + a] = S_orig[nS * o + a];
    }
    double *M = calloc((size_t)nc * nM, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < nc; ++c)
        if (t->nchild[c] == 0)
            orc_p2m_orders(s_lo, s_hi, pt, t->centre + 3 * c, t->end[c] - t->begin[c],
                           pos + 3 * t->begin[c], S + nS * t->begin[c], M + (size_t)nM * c);
    for (int l = t->nlevels - 2; l >= 0; --l) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t c = t->level_begin[l]; c < t->level_begin[l + 1]; ++c)
            for (int i = 0; i < t->nchild[c]; ++i) {
                int64_t ch = t->child_first[c] + i;
                orc_m2m(s, pt, t->centre + 3 * ch, t->centre + 3 * c, M + (size_t)nM * ch,
                        M + (size_t)nM * c);
            }
    }
    int64_t *rank = malloc(sizeof(int64_t) * n);
    for (int64_t k = 0; k < n; ++k) rank[t->perm[k]] = k;
    bh_ctx b = {t, pos, S, M, s, s_hi, p, nM, nS, theta * theta};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < ntarget; ++q) {
        int64_t k = rank[targets ? targets[q] : q];
        double f = 0.0, g[3] = {0.0, 0.0, 0.0};
        bh_walk(&b, 0, k, pos + 3 * k, &f, g);
        phi[q] = f;
        E[3 * q] = -g[0]; E[3 * q + 1] = -g[1]; E[3 * q + 2] = -g[2];
    }
    free(pos); free(S); free(M); free(rank);
    return 0;
}

int orc_bh(const orc_tree *t, const double *pos_orig, int s, int p, const double *S_orig,
           double theta, int64_t ntarget, const int64_t *targets, double *phi, double *E)
{
    return orc_bh_orders(t, pos_orig, s, s, p, S_orig, theta, ntarget, targets, phi, E);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
