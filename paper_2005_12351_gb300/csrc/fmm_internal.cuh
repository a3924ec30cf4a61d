// fmm_internal.cuh -- shared declarations of the sm_103a FMM library.
//
// Layout in device memory (one system):
//   particles, Morton-sorted: px/py/pz [n] f64 (SoA), S [n x nS] f64, perm [n] i32
//   cells, breadth-first:     level/parent/child_first/nchild/begin/end/cx,cy,cz (i32)
//                             centre [ncells x 3] f64, half [ncells] f64
//   expansions:               M [ncells x nM] f64, L [ncells x nL] f64 (row per cell)
//   lists (CSR by target):    m2l_src/m2l_didx [n_m2l], m2l_off [ncells+1]
//                             p2p_src [n_p2p], p2p_off [ncells+1]
//   derivative tables:        D [n_doffsets x ntot(p+s)] f64
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fmm_gb300.h"

namespace fmm {

constexpr int kLevels = 21;            // key depth: 3 x 21 = 63 bits
constexpr int kMaxOrder = 16;          // multi-index tables cover |n| <= 16
constexpr int kMaxTot = 969;           // ntot(16)
constexpr int kKeyBias = 1 << 16;      // D-table key: offsets in [-2^16, 2^16)

// device error word bits
constexpr int kErrNonFinite = 1;
constexpr int kErrKeyRange = 2;
constexpr int kErrHashFull = 4;
constexpr int kErrTcTimeout = 8;       // a tensor-core M2L wait gave up (word 1 of b_err)
constexpr int kErrSortWait = 16;       // a look-back wait of the radix sort gave up
constexpr int kErrLongRow = 32;        // a row of an interaction list too long for the row sort

inline int ntot(int p) { return p < 0 ? 0 : (p + 1) * (p + 2) * (p + 3) / 6; }
inline int nshell(int k) { return (k + 1) * (k + 2) / 2; }

// Multi-index enumeration of the library (graded lexicographic, §3.1 of the
// paper): shell by shell; inside a shell, by increasing ny + nz, then by
// increasing nz.  Built once by enumeration into a lookup cube.
struct MultiIndex {
    int nx[kMaxTot], ny[kMaxTot], nz[kMaxTot];
    int16_t lut[kMaxOrder + 1][kMaxOrder + 1][kMaxOrder + 1];
    MultiIndex();
    int operator()(int x, int y, int z) const { return lut[x][y][z]; }
};
const MultiIndex &multi_index();

// Host-built operator tables for one (s, p) pair, uploaded once per change.
struct OpTables {
    int s = -1, p = -1, n_lo = -1;
    int nS = 0, nM = 0, nL = 0, nD = 0, m0 = 0;
    // P2M: for each m (0..nM), up to nS terms (a, mono index of m - a); -1 = none
    std::vector<int> p2m_terms;          // [nM x nS] mono index or -1
    // monomial recurrences: mono[k] = mono[par[k]] * d[axis[k]] / k_axis
    std::vector<int> mono_par, mono_axis, mono_pow;   // [ntot(P)]
    // M2M: CSR over outputs n (M storage), terms (mono k, M index q)
    std::vector<int> m2m_off, m2m_k, m2m_q;
    // L2L: CSR over outputs n (L storage), terms (mono k, L index n+k)
    std::vector<int> l2l_off, l2l_k, l2l_q;
    // L2P gradient: for |k| <= p-1, L index of k + e_d (3 per k)
    std::vector<int> l2p_grad;
    // M2L: per-thread term lists (slot-major) and the partial-sum reduction map
    int m2l_threads = 0, m2l_T = 0, m2l_slots = 0;
    std::vector<uint32_t> m2l_desc;      // [T x threads]
    std::vector<int> m2l_red_off, m2l_red_src;   // CSR over n: partial slot ids
    // Harmonic M2L (D_k = grad^k 1/r is traceless: D_{k+2x} + D_{k+2y} + D_{k+2z} = 0).
    // The M2L terms then run over the m with m_z <= 1 of the folded multipole M'
    // and the n with n_z <= 1; the other L_n follow from the same identity.
    bool harmonic = false;
    int nMh = 0;                         // m kept: storage index h_rm[r], graded order
    std::vector<int> h_rm;
    // fold: (t, a, b) per entry, M'_t = M_t - M'_a - M'_b (a, b = t - 2x + 2z,
    // t - 2y + 2z; -1 absent), levels of decreasing t_z, CSR over levels
    std::vector<int> h_fold, h_fold_off;
    // unfold: (n, a, b), L_n = -L_a - L_b (a, b = n + 2x - 2z, n + 2y - 2z),
    // levels of increasing n_z >= 2, CSR over levels
    std::vector<int> h_unfold, h_unfold_off;
    // stored local components: nLh per cell, the n with n_z <= 1 (graded order)
    // when harmonic, all nL otherwise; h_rn[r] = full index of stored slot r
    int nLh = 0;
    std::vector<int> h_rn;
};
// s: the lowest source order (the expansion's), s_hi: the highest (mixed
// systems carry every order s..s_hi per particle; P2M reads all of them)
void build_tables(OpTables &T, int s, int s_hi, int p, int n_lo, int m2l_threads, bool harmonic);

// Operator layout of the tensor-core M2L (FMM_3XTF32) for one (s, p).  The
// local-expansion columns are cut into groups of at most 128 (width W); the
// multipoles into K-blocks of 8, each reaching N <= W columns of a group (a
// multiple of 16).  A key's operator image holds, per (group, K-block), a
// 32-byte-swizzled tile of W + N rows: the hi halves of rows 0..N-1, zero
// rows up to W, then the lo halves.  Per image float: the D entry it takes
// (d | |n+m| << 16 | (|m|-s) << 24, -1 for zero) and its byte position
// (offset | 1 << 30 for a lo half).
struct TcLayout {
    int s = -1, p = -1, nkb = 0, Np = 0, ngroups = 0, E = 0, b_stage = 0, img_bytes = 0;
    // h = 1: the harmonic M2L (K over the kept m of the folded multipole,
    // columns over the n with n_z <= 1); col_n = full local index per column
    int h = -1, ncol = 0;
    std::vector<int> col_n;
    int g_width[2] = {0, 0}, g_nkb[2] = {0, 0}, g_nkc[2] = {0, 0};
    std::vector<int> kb_n;        // [nkb] columns a K-block reaches (from column 0)
    std::vector<int> img_off;     // [2 x (nkb + 1)] byte offset of block (g, kb) in an image
    std::vector<int> el_src, el_pos;
};

// Layout of the tiled SIMT FP32 M2L (m2l32_tile.cu): the kept locals n with
// |n| >= n_lo in graded order as columns, in blocks of 8; block b takes the
// first mb[b] kept multipoles m (a multiple of 4, graded order: those that
// reach its lowest-order column, rounded up), and a key's operator image holds,
// from float boff[b] on, T[8 b + j][m] at 8 m + j (zero outside the
// truncation).  el_src: per image float, the D entry | order << 16 |
// (|m| - s) << 24, or -1 for a zero.
struct T32Layout {
    int s = -1, p = -1, h = -1, n_lo = -1, nM = 0, ncol = 0, nb = 0, Np = 0, E = 0;
    std::vector<int> col_n, mb, boff, el_src;
};

// threads of the M2L blocks (the per-thread term lists are built for it)
constexpr int kM2LThreadsShared = 128;

// Device views of the uploaded tables (passed to kernels by value).
struct DevTables {
    int s, p, n_lo, nS, nM, nL, nD, m0, nK, nG;
    const int *p2m_terms;
    const int *m2m_off, *m2m_k, *m2m_q;
    const int *l2l_off, *l2l_k, *l2l_q;
    const int *l2p_grad;
    const int *m2l_red_off, *m2l_red_src;
    const uint32_t *m2l_desc;
    int m2l_T, m2l_slots;
    // packed multi-indices nx | ny << 5 | nz << 10 | |n| << 15 (global memory:
    // lanes may index it divergently, which the constant cache would serialise)
    const int *mi;
    // harmonic M2L (OpTables): nMh = nM and no levels when off
    int harmonic, nMh, h_fold_lev, h_unfold_lev;
    const int *h_rm, *h_fold, *h_fold_off, *h_unfold, *h_unfold_off;
    // stored local components (OpTables): nLh per cell, slot r holds L_{h_rn[r]}
    int nLh;
    const int *h_rn;
};

// A cell's full local expansion in shared memory (Lf[nL]) from its stored row:
// the stored components, then -- harmonic storage -- the others in increasing
// n_z from the trace identity L_n = -L_{n+2x-2z} - L_{n+2y-2z} (§3.1: 1/r is
// harmonic, so are the local expansions of its M2L and their L2L shifts).
// Called by every thread of the block; ends with a barrier.
template <typename T, bool CG = false>
__device__ __forceinline__ void expand_local(const T *row, const DevTables &tb, T *Lf)
{
    for (int r = threadIdx.x; r < tb.nLh; r += blockDim.x) Lf[tb.h_rn[r]] = CG ? __ldcg(row + r) : row[r];
    for (int l = 0; l < tb.h_unfold_lev; ++l) {
        __syncthreads();
        for (int q = tb.h_unfold_off[l] + threadIdx.x; q < tb.h_unfold_off[l + 1]; q += blockDim.x)
            Lf[tb.h_unfold[3 * q]] = -Lf[tb.h_unfold[3 * q + 1]] - Lf[tb.h_unfold[3 * q + 2]];
    }
    __syncthreads();
}

// the same, for a row another block of the same launch may have written (the
// loads bypass the incoherent L1)
template <typename T>
__device__ __forceinline__ void expand_local_cg(const T *row, const DevTables &tb, T *Lf)
{
    expand_local<T, true>(row, tb, Lf);
}

// Bounded wait of thread 0 of a block for a flag another block of the same
// launch sets; false if it gave up (about a second).  The caller orders the
// wait before its reads with a fence.
__device__ __forceinline__ bool wait_flag(const unsigned *flag)
{
    const volatile unsigned *f = flag;
    if (*f) return true;
    const long long t0 = clock64();
    while (!*f) {
        if (clock64() - t0 > (1ll << 31)) return false;
        __nanosleep(32);
    }
    return true;
}

__device__ __forceinline__ int mi_at(const int *mi, int k) { return __ldg(mi + k); }
__device__ __forceinline__ int mi_nx(int v) { return v & 31; }
__device__ __forceinline__ int mi_ny(int v) { return (v >> 5) & 31; }
__device__ __forceinline__ int mi_nz(int v) { return (v >> 10) & 31; }
__device__ __forceinline__ int mi_shell(int v) { return v >> 15; }

}  // namespace fmm

// ---------------------------------------------------------------------------
// The handle.
// ---------------------------------------------------------------------------
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct fmm_tree {
    int device = 0;
    cudaStream_t stream = nullptr;
    int max_leaf = 64;
    fmm_precision prec = FMM_FP64;
    size_t budget = 0;
    size_t held = 0;
    std::string err;
    int64_t launches = 0;
    // allocation-failure injection (FMM_FAIL_ALLOC at create): the fail_alloc_at-th
    // device allocation of the handle fails once; 0 = off
    int64_t alloc_count = 0, fail_alloc_at = 0;

    // system
    int64_t n = 0;
    // source orders s..s_hi per particle (s_hi = s: one order); nS moments each
    int s = -1, s_hi = -1, nS = 0;
    bool have_sources = false;
    int64_t ncells = 0, nleaves = 0;
    int nlevels = 0;
    std::vector<int> level_begin;          // host copy, nlevels + 1
    double lo[3] = {0, 0, 0}, side = 1.0;  // root box of system 0
    std::vector<int64_t> sys_off;          // host: system s owns particles [off[s], off[s+1])
    std::vector<double> sys_box;           // host copy: (lo_x, lo_y, lo_z, side) per system

    // lists
    double theta = 0.0;
    bool have_lists = false;
    int64_t n_m2l = 0, n_p2p = 0, n_p2p_inter = 0, n_doff = 0;
    size_t m2l_cap_hint = 0;
    int max_gap = 0;                       // largest level gap of an M2L pair
    // D tables / operator tables
    int d_p = -1;                          // p the D table was built for
    fmm::OpTables tab;
    int tab_key_s = -1, tab_key_p = -1, tab_key_nlo = -1, tab_key_h = -1, tab_key_shi = -1;
    int64_t m_cells = 0;                   // rows of the M/L buffers as sized

    // profiling
    bool profiling = false;
    cudaEvent_t ev[fmm::kLevels + 16];
    bool ev_made = false;
    float phase_ms[FMM_NUM_PHASES];

    // device buffers (all owned)
    DevBuf b_err, b_box;
    DevBuf b_keys, b_keys2, b_idx, b_idx2, b_hist;
    DevBuf b_px, b_py, b_pz, b_S, b_perm;
    DevBuf b_level, b_parent, b_child, b_nchild, b_begin, b_end, b_cx, b_cy, b_cz, b_sys;
    DevBuf b_sysoff, b_sysbox, b_syseside;
    // log2 of each system's root side (device int array)
    const int *sys_eside_dev() const { return (const int *)b_syseside.ptr; }
    DevBuf b_centre, b_half, b_leaves;
    DevBuf b_flags, b_scan, b_scan_tmp;
    DevBuf b_ctl;                          // level counts of the cell build
    DevBuf b_ud;                           // upward arrival counters, downward flags
    DevBuf b_front, b_front2, b_m2l_raw, b_p2p_raw, b_counters;
    DevBuf b_tcell;                        // packed cell records of the traversal
    DevBuf b_rows, b_m2l_slot, b_p2p_slot, b_long;   // row counts, positions in rows, long rows
    DevBuf b_m2l_src, b_m2l_off, b_m2l_didx, b_p2p_src, b_p2p_off, b_lkeys, b_lkeys2, b_lval, b_lval2;
    DevBuf b_hash, b_dkeys, b_D;
    DevBuf b_dsort, b_dsort_h;             // scratch of the canonical D-key numbering
    DevBuf b_M, b_L, b_phi, b_E;
    DevBuf b_Mh, b_Mh32;                   // folded multipoles of the harmonic M2L
    // Barnes-Hut: the M2P term table of (bh_key_s, bh_key_p)
    int bh_key_s = -1, bh_key_p = -1;      // bh_key_s: key of the program in b_bh_mt
    int bh_nD = 0, bh_nmt = 0, bh_ncoef = 0;
    bool bh_ran = false;                   // b_bh_cnt holds the last walk's counts
    DevBuf b_bh_mt, b_bh_cnt;
    DevBuf b_tab_i32, b_tab_u32;
    // mixed-precision state
    DevBuf b_o32, b_S32, b_M32, b_L32, b_D32;
    // request staging (serving): host inputs and outputs pass through these
    DevBuf b_req_in, b_req_out;
    int d32_p = -1;                        // p the FP32 D table was built for
    // tensor-core M2L (FMM_3XTF32): target tiles, their key rows and chunks,
    // derived from the lists; operator images derived from the D table
    bool tc_plan = false;
    int tc_img_p = -1, tc_sms = 0;
    int64_t tc_T = 0, tc_tiles = 0, tc_W = 0, tc_rows = 0, tc_chunks = 0;
    int tc_G = 0;                          // key rows per chunk
    fmm::TcLayout tc_lay;
    DevBuf b_tc_keys, b_tc_keys2, b_tc_vals, b_tc_vals2, b_tc_hist, b_tc_scan, b_tc_cnt;
    DevBuf b_tc_tgt, b_tc_bits, b_tc_wpre, b_tc_rcnt, b_tc_ccnt, b_tc_roff, b_tc_coff;
    DevBuf b_tc_rowkey, b_tc_crb, b_tc_cre, b_tc_slot, b_tc_el, b_tc_img, b_tc_part;
    // tiled SIMT FP32 M2L on the same plan: its layout, FP32 operator images
    // (m32_img_p: p they were built for, -1 none) and their element map
    fmm::T32Layout m32_lay;
    int m32_img_p = -1;
    DevBuf b_m32_el, b_m32_img;

    // symmetric FP64 P2P (p2p_variant 2), derived from the lists: per list
    // entry its mirror entry (-1: none) and, for an entry (A, B) with B > A,
    // the first of B's rows in the reverse-term buffer; sym_rows = total rows
    // (-1: more than the 32-bit row index covers)
    bool sym_plan = false;
    int64_t sym_rows = 0;
    DevBuf b_sym_mir, b_sym_cnt, b_sym_base, b_sym_scan, b_sym_tot, b_sym_rev, b_sym_fwd;

    // tuning (fmm_autotune, fmm_set_tuning; defaults otherwise): FP64 P2P kernel
    // (0 one target per thread, 1 two, 2 each leaf pair once for both
    // directions), FMM_3XTF32 M2L on the SIMT FP32 kernel instead of the
    // tensor cores, rows per chunk of the tensor-core M2L (tc_G above)
    int p2p_variant = 2;
    int p2p_tt = 2;                        // FP32 forms' one-way P2P: targets per thread (1 or 2)
    bool m2l_simt = false;
    bool m2l_tiled = true;                 // SIMT FP32 M2L over the plan's tiles (else per target cell)
    bool m2l_harmonic = true;              // SIMT M2L over the traceless components
    bool tuned = false;
    // fmm_evaluate_graph: the evaluate of one parameter set captured as a CUDA graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    // side stream of the mixed forms (the M2L plan is built on it while the
    // upward pass runs) and the two events that join it to the handle's stream
    cudaStream_t side_st = nullptr;
    cudaEvent_t ev_lists = nullptr, ev_plan = nullptr;
    int g_p = -1, g_phi = 0, g_field = 0;
    double g_theta = 0.0;
    double *g_pot = nullptr, *g_fld = nullptr;
};

// ---------------------------------------------------------------------------
// Internal host API (implemented in the .cu files; all enqueue on `st`).
// ---------------------------------------------------------------------------
namespace fmm {

fmm_status ensure(fmm_tree *t, DevBuf &b, size_t bytes);
void release(fmm_tree *t, DevBuf &b);
fmm_status cuda_check(fmm_tree *t, cudaError_t e, const char *what);

// primitives.cu
size_t scan_scratch_bytes(int64_t n);
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *scratch,
                        cudaStream_t st, int64_t *launches);
// Scratch of radix_sort_pairs in 32-bit words: digit counts of up to 8
// passes and 16 tile counters (kRadixHead words), then two areas of 256
// 64-bit status words per tile of 4096 keys.
constexpr int kRadixMaxPasses = 8;
constexpr int kRadixTile = 4096;       // keys per one-sweep tile
constexpr int64_t kRadixHead = kRadixMaxPasses * 256 + 16;
constexpr int64_t radix_hist_words(int64_t n)
{
    return kRadixHead + 4 * 256 * ((n + kRadixTile - 1) / kRadixTile > 0 ? (n + kRadixTile - 1) / kRadixTile : 1);
}
size_t radix_hist_bytes(int64_t n);
// Stable LSD radix sort of (key, value) pairs on bits [0, end_bit), end_bit
// <= 64, n < 2^32.  The result ends in (keys, vals); (keys2, vals2) are
// scratch of the same size, hist holds radix_hist_bytes(n).  A bounded wait
// of the one-sweep passes that gave up sets kErrSortWait in *err (device).
// counted: the digit counts of every pass are already in hist and the first
// status area is zero (the caller's key kernel formed them, after zeroing
// the kRadixHead head words), so the sort skips its counting launch.
void radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys2, uint32_t *vals2, int64_t n,
                      int end_bit, uint32_t *hist, int *err, cudaStream_t st, int64_t *launches,
                      bool counted = false);

// Per-device set-up of the sort (its kernels loaded, the scatter's shared-
// memory limit raised); radix_sort_pairs calls it, and callers that must not
// trigger module loading later call it ahead of time.
void radix_sort_prepare();

// tree.cu
fmm_status build_tree(fmm_tree *t, const double *pos, const double *mom);
fmm_status build_lists(fmm_tree *t, double theta);
// loads the Morton-order kernels on the current device (no launch)
void morton_order_prepare();
fmm_status morton_order_raw(cudaStream_t st, const double *pos, int64_t n, uint64_t *keys,
                            uint32_t *idx, uint64_t *keys2, uint32_t *idx2, uint32_t *hist,
                            unsigned long long *box_scratch, double *box_out, int *err,
                            int64_t *launches);

// operators.cu
fmm_status upload_tables(fmm_tree *t, int s, int p, int n_lo, DevTables *dt, const int32_t **lut);
fmm_status build_dtables(fmm_tree *t, int p, const DevTables &tb, const int32_t *lut);
fmm_status run_expansions(fmm_tree *t, int p, int want_phi, int want_field);
// P2M + M2M of the tables' (s, p) into b_M; rec: record the phase events
fmm_status run_upward(fmm_tree *t, const DevTables &tb, bool rec);
// bh.cu: multipolar Barnes-Hut of order p (multipoles s <= |m| <= p), FP64
fmm_status run_bh(fmm_tree *t, int p, double theta, int want_phi, int want_field, double *phi_out,
                  double *E_out);
// M' of the harmonic M2L for every cell: Mh[c][r] = fold(M[c])[h_rm[r]]
void launch_fold_m(cudaStream_t st, const double *M, int ldM, int64_t nc, const DevTables &tb,
                   double *Mh, int ldH);
void launch_fold_m(cudaStream_t st, const float *M, int ldM, int64_t nc, const DevTables &tb,
                   float *Mh, int ldH);
// mixed.cu (FMM_FP32): scaled FP32 expansions, FP32 pair arithmetic, FP64 outputs
fmm_status run_mixed(fmm_tree *t, int p, int want_phi, int want_field, double *phi_out,
                     double *E_out);
// m2l_tc.cu: whether the tensor-core M2L covers (s, p) (fills t->tc_lay), and
// the M2L of the mixed-precision form on it: M and L are the scaled FP32
// expansions, L zeroed by the caller
bool tc_usable(fmm_tree *t, int s, int p);
// builds the plan, the operator images and the partial buffer for p (FMM_EBUDGET
// when they do not fit the handle's budget); tc_release frees all of it
fmm_status tc_prepare(fmm_tree *t, int p);
void tc_release(fmm_tree *t);
// (M: folded multipoles, nM = tb.nMh columns, when the handle's M2L is harmonic;
// tb supplies the unfold of L)
fmm_status run_m2l_tc(fmm_tree *t, int p, const float *M, int ldM, int nM, int nL,
                      const DevTables &tb, float *L);
// the plan alone (target tiles, key rows, chunks, source slots; one host sync),
// and the double-float sum of the chunk partials [chunks][128][Np] into the stored
// locals of the tiles' targets (NaN where err holds a tensor-core timeout)
fmm_status tc_build_plan(fmm_tree *t);
void launch_tc_reduce(fmm_tree *t, int Np, int ncol, const int32_t *col_n, int nL, const DevTables &tb,
                      const unsigned *err, float *L);
// m2l32_tile.cu: the SIMT FP32 M2L over the same plan, one thread per target
// of a tile, the key's operator read by the whole block.  Usable when the
// layout for (s, p, harmonic, n_lo) fits (fills t->m32_lay); prepare builds
// the plan, images and partials (FMM_EBUDGET over the handle's budget)
bool m32_usable(fmm_tree *t, int s, int p, int harmonic, int n_lo);
fmm_status m32_prepare(fmm_tree *t, int p);
fmm_status run_m2l32_tile(fmm_tree *t, int p, const float *M, int ldM, const DevTables &tb, float *L);
// api.cu: the handle's side stream and join events, created on first use
fmm_status side_stream(fmm_tree *t);
// api.cu: the compute of an evaluate whose lists are current (no host sync)
fmm_status evaluate_body(fmm_tree *t, int p, int want_phi, int want_field, double *phi, double *E);
// graph.cu: drop a captured evaluate graph (the tree or the tuning changed)
void drop_graph(fmm_tree *t);
// p2p.cu
fmm_status run_p2p(fmm_tree *t, int want_phi, int want_field, double *phi_out, double *E_out);
// the symmetric P2P's plan (mirror entries, reverse-row offsets; one host sync
// when built) and its buffers for NC output components (rows of NC doubles, or
// of NC floats in the FP32 forms); FMM_EBUDGET over the handle's budget
fmm_status sym_prepare(fmm_tree *t, int NC);
void launch_check_rsqrt(cudaStream_t st, const double *x, int64_t n, double *own, double *ref);
// m2l_tc.cu
fmm_status check_umma(cudaStream_t st, const float *A, const float *B, float *D, int nkb, int N,
                      const int *kbn, int a_tmem, int passes, unsigned *err);
void launch_direct(cudaStream_t st, const double *pos, const double *mom, int64_t n, int s, int s_hi,
                   const int32_t *targets, int64_t nt, double *phi, double *E, int64_t *launches);

}  // namespace fmm

namespace fmm {
// Streaming multiprocessors of the current device (grid caps of the
// grid-stride kernels scale with it); 1 if the query fails.
inline int sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return 1;
    }
    return sms;
}

// Raises a kernel's dynamic shared-memory limit to the most a block can take
// next to its static shared memory.  The value depends only on the kernel, so
// handles that launch it concurrently from several threads never lower the
// limit under one another's launches (a per-launch size would race).
template <typename K>
inline void allow_max_dynamic_smem(K kern)
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}
}  // namespace fmm

#define FMM_TRY(expr)                         \
    do {                                      \
        fmm_status _st = (expr);              \
        if (_st != FMM_OK) return _st;        \
    } while (0)
