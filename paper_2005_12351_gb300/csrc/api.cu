// api.cu -- the extern "C" boundary declared in include/fmm_gb300.h.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

fmm_status cuda_check(fmm_tree *t, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return FMM_OK;
    if (t) t->err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? FMM_ENOMEM : FMM_ECUDA;
}

void all_buffers(fmm_tree *t, std::vector<DevBuf *> &v)
{
    DevBuf *b[] = {&t->b_req_in, &t->b_req_out, &t->b_sys, &t->b_sysoff, &t->b_sysbox,
                   &t->b_syseside, &t->b_o32, &t->b_S32,
                   &t->b_M32, &t->b_L32, &t->b_D32, &t->b_err, &t->b_box, &t->b_keys, &t->b_keys2, &t->b_idx, &t->b_idx2,
                   &t->b_hist, &t->b_px, &t->b_py, &t->b_pz, &t->b_S, &t->b_perm, &t->b_level,
                   &t->b_parent, &t->b_child, &t->b_nchild, &t->b_begin, &t->b_end, &t->b_cx,
                   &t->b_cy, &t->b_cz, &t->b_centre, &t->b_half, &t->b_leaves, &t->b_flags,
                   &t->b_scan, &t->b_scan_tmp, &t->b_front, &t->b_front2, &t->b_m2l_raw,
                   &t->b_p2p_raw, &t->b_counters, &t->b_tcell, &t->b_rows, &t->b_m2l_slot,
                   &t->b_p2p_slot, &t->b_long, &t->b_m2l_src, &t->b_m2l_off, &t->b_m2l_didx,
                   &t->b_p2p_src, &t->b_p2p_off, &t->b_lkeys, &t->b_lkeys2, &t->b_lval,
                   &t->b_lval2, &t->b_hash, &t->b_dkeys, &t->b_dsort, &t->b_dsort_h, &t->b_D, &t->b_M, &t->b_L, &t->b_phi,
                   &t->b_E, &t->b_tab_i32, &t->b_tab_u32, &t->b_tc_keys, &t->b_tc_keys2,
                   &t->b_tc_vals, &t->b_tc_vals2, &t->b_tc_hist, &t->b_tc_scan, &t->b_tc_cnt,
                   &t->b_tc_tgt, &t->b_tc_bits, &t->b_tc_wpre, &t->b_tc_rcnt, &t->b_tc_ccnt,
                   &t->b_tc_roff, &t->b_tc_coff, &t->b_tc_rowkey, &t->b_tc_crb, &t->b_tc_cre,
                   &t->b_tc_slot, &t->b_tc_el, &t->b_tc_img, &t->b_tc_part, &t->b_m32_el, &t->b_m32_img,
                   &t->b_sym_mir,
                   &t->b_sym_cnt, &t->b_sym_base, &t->b_sym_scan, &t->b_sym_tot, &t->b_sym_rev,
                   &t->b_sym_fwd, &t->b_Mh, &t->b_Mh32, &t->b_bh_mt, &t->b_bh_cnt, &t->b_ctl, &t->b_ud};
    v.assign(b, b + sizeof(b) / sizeof(b[0]));
}

// After a failed allocation the buffer being grown is gone (ensure releases it
// first), and with it whatever state lived there.  The handle goes back to the
// state of a fresh one (keeping its tuning): every buffer but the error word
// and the box scratch released, the tree, the lists, the captured graph and
// every cache keyed on them dropped, so that no later call reads a buffer that
// is not there.  fmm_set_sources rebuilds all of it.
static void forget_state(fmm_tree *t)
{
    drop_graph(t);
    std::vector<DevBuf *> v;
    all_buffers(t, v);
    for (DevBuf *b : v)
        if (b != &t->b_err && b != &t->b_box) release(t, *b);
    t->have_sources = false;
    t->have_lists = false;
    t->tc_plan = false;
    t->tc_img_p = -1;
    t->m32_img_p = -1;
    t->sym_plan = false;
    t->bh_ran = false;
    t->bh_key_s = -1;
    t->d_p = -1;
    t->d32_p = -1;
    t->tab_key_s = t->tab_key_p = t->tab_key_nlo = t->tab_key_h = t->tab_key_shi = -1;
}

fmm_status side_stream(fmm_tree *t)
{
    if (!t->side_st)
        FMM_TRY(cuda_check(t, cudaStreamCreateWithFlags(&t->side_st, cudaStreamNonBlocking), "stream"));
    if (!t->ev_lists)
        FMM_TRY(cuda_check(t, cudaEventCreateWithFlags(&t->ev_lists, cudaEventDisableTiming), "event"));
    if (!t->ev_plan)
        FMM_TRY(cuda_check(t, cudaEventCreateWithFlags(&t->ev_plan, cudaEventDisableTiming), "event"));
    return FMM_OK;
}

fmm_status ensure(fmm_tree *t, DevBuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return FMM_OK;
    bytes = (bytes + 255) & ~(size_t)255;
    if (t->budget && t->held - b.bytes + bytes > t->budget) {
        t->err = "device memory budget exceeded (" + std::to_string(t->held - b.bytes + bytes) +
                 " > " + std::to_string(t->budget) + " bytes)";
        return FMM_EBUDGET;
    }
    release(t, b);
    void *p = nullptr;
    const bool injected = t->fail_alloc_at > 0 && ++t->alloc_count == t->fail_alloc_at;
    cudaError_t e = injected ? cudaErrorMemoryAllocation : cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        if (!injected) cudaGetLastError();
        t->err = "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e) +
                 (injected ? " (injected by FMM_FAIL_ALLOC)" : "");
        forget_state(t);
        return FMM_ENOMEM;
    }
    b.ptr = p;
    b.bytes = bytes;
    t->held += bytes;
    return FMM_OK;
}

void release(fmm_tree *t, DevBuf &b)
{
    if (b.ptr) {
        // work already queued on the handle's stream may still read this buffer
        // (a grow copy, an earlier kernel): once freed, another handle's
        // allocation on another stream may receive the same memory
        if (t->stream) cudaStreamSynchronize(t->stream);
        else cudaDeviceSynchronize();
        cudaFree(b.ptr);
        t->held -= b.bytes;
    }
    b.ptr = nullptr;
    b.bytes = 0;
}

}  // namespace fmm

namespace fmm {

fmm_status evaluate_body(fmm_tree *t, int p, int want_phi, int want_field, double *phi, double *E)
{
    if (t->prec == FMM_FP32 || t->prec == FMM_3XTF32)
        return run_mixed(t, p, want_phi, want_field, phi, E);
    FMM_TRY(run_expansions(t, p, want_phi, want_field));
    return run_p2p(t, want_phi, want_field, phi, E);
}

}  // namespace fmm

using namespace fmm;

namespace {

thread_local std::string g_create_err;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

void record(fmm_tree *t, int i)
{
    if (t->profiling) cudaEventRecord(t->ev[i], t->stream);
}


fmm_status fail(fmm_tree *t, fmm_status s, const std::string &msg)
{
    if (t) t->err = msg;
    return s;
}

}  // namespace

extern "C" {

const char *fmm_status_string(fmm_status s)
{
    switch (s) {
    case FMM_OK: return "ok";
    case FMM_EINVAL: return "invalid argument";
    case FMM_ENOMEM: return "out of device memory";
    case FMM_EORDER: return "expansion order out of range";
    case FMM_ECUDA: return "CUDA error";
    case FMM_ETIMEOUT: return "device wait timed out";
    case FMM_EBUDGET: return "device memory budget exceeded";
    case FMM_ESTATE: return "call out of order";
    }
    return "unknown status";
}

const char *fmm_last_error(const fmm_tree *t)
{
    return t ? t->err.c_str() : g_create_err.c_str();
}

fmm_status fmm_create_tree(fmm_tree **out, int device, void *cuda_stream, int max_leaf,
                           fmm_precision prec, size_t mem_budget_bytes)
{
    g_create_err.clear();
    if (!out) { g_create_err = "out is NULL"; return FMM_EINVAL; }
    *out = nullptr;
    if (max_leaf < 1) { g_create_err = "max_leaf must be >= 1"; return FMM_EINVAL; }
    if (prec != FMM_FP64 && prec != FMM_FP32 && prec != FMM_3XTF32) {
        g_create_err = "unknown precision";
        return FMM_EINVAL;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        g_create_err = "no CUDA device " + std::to_string(device);
        return FMM_EINVAL;
    }
    DeviceGuard g(device);
    fmm_tree *t = new (std::nothrow) fmm_tree();
    if (!t) { g_create_err = "host allocation failed"; return FMM_ENOMEM; }
    t->device = device;
    t->stream = (cudaStream_t)cuda_stream;
    t->max_leaf = max_leaf;
    t->prec = prec;
    // the symmetric near field pays off where pairs are FP64; the FP32 forms'
    // pairs are cheap next to its warp sums, so they start one-way
    t->p2p_variant = prec == FMM_FP64 ? 2 : 1;
    t->budget = mem_budget_bytes;
    if (const char *env = getenv("FMM_FAIL_ALLOC")) t->fail_alloc_at = std::max(0ll, atoll(env));
    std::memset(t->phase_ms, 0, sizeof(t->phase_ms));
    fmm_status st = ensure(t, t->b_err, 16);
    if (st == FMM_OK) st = ensure(t, t->b_box, 256);
    if (st == FMM_OK) st = cuda_check(t, cudaMemsetAsync(t->b_err.ptr, 0, 16, t->stream), "memset");
    if (st != FMM_OK) {
        g_create_err = t->err;
        fmm_destroy(t);
        return st;
    }
    *out = t;
    return FMM_OK;
}

fmm_status fmm_destroy(fmm_tree *t)
{
    if (!t) return FMM_OK;
    DeviceGuard g(t->device);
    if (t->stream) cudaStreamSynchronize(t->stream);
    else cudaDeviceSynchronize();
    drop_graph(t);
    if (t->cap_stream) cudaStreamDestroy(t->cap_stream);
    if (t->side_st) {
        cudaStreamSynchronize(t->side_st);
        cudaStreamDestroy(t->side_st);
    }
    if (t->ev_lists) cudaEventDestroy(t->ev_lists);
    if (t->ev_plan) cudaEventDestroy(t->ev_plan);
    std::vector<DevBuf *> v;
    all_buffers(t, v);
    for (DevBuf *b : v) release(t, *b);
    if (t->ev_made)
        for (auto &ev : t->ev) cudaEventDestroy(ev);
    delete t;
    return FMM_OK;
}

fmm_status fmm_set_profiling(fmm_tree *t, int enable)
{
    if (!t) return FMM_EINVAL;
    DeviceGuard g(t->device);
    if (enable && !t->ev_made) {
        for (auto &ev : t->ev)
            if (cudaEventCreate(&ev) != cudaSuccess) return fail(t, FMM_ECUDA, "event create");
        t->ev_made = true;
    }
    t->profiling = enable != 0;
    return FMM_OK;
}

fmm_status fmm_get_phase_times(const fmm_tree *t, float *ms_out)
{
    if (!t || !ms_out) return FMM_EINVAL;
    std::memcpy(ms_out, t->phase_ms, sizeof(t->phase_ms));
    return FMM_OK;
}

int64_t fmm_launch_count(const fmm_tree *t) { return t ? t->launches : -1; }

static fmm_status set_sources_impl(fmm_tree *t, const double *positions, const double *moments,
                                   int64_t n, int source_order, int source_order_hi);

fmm_status fmm_set_sources(fmm_tree *t, const double *positions, const double *moments, int64_t n,
                           int source_order)
{
    if (!t) return FMM_EINVAL;
    t->err.clear();
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(t, FMM_EINVAL, "n out of range");
    t->sys_off.assign({0, n});
    return set_sources_impl(t, positions, moments, n, source_order, source_order);
}

fmm_status fmm_set_sources_mixed(fmm_tree *t, const double *positions, const double *moments,
                                 int64_t n, int s_lo, int s_hi)
{
    if (!t) return FMM_EINVAL;
    t->err.clear();
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(t, FMM_EINVAL, "n out of range");
    if (s_lo < 0 || s_hi < s_lo || s_hi > FMM_MAX_SOURCE_ORDER)
        return fail(t, FMM_EORDER, "need 0 <= s_lo <= s_hi <= 2");
    if (s_hi > s_lo && t->prec != FMM_FP64)
        return fail(t, FMM_EORDER, "mixed source orders are evaluated by the FP64 form");
    t->sys_off.assign({0, n});
    return set_sources_impl(t, positions, moments, n, s_lo, s_hi);
}

fmm_status fmm_set_sources_batch(fmm_tree *t, const double *positions, const double *moments,
                                 const int64_t *offsets, int count, int source_order)
{
    if (!t) return FMM_EINVAL;
    t->err.clear();
    if (count < 1 || count > (1 << 24) || !offsets)
        return fail(t, FMM_EINVAL, "count must be in [1, 2^24] with a host offsets array");
    if (offsets[0] != 0) return fail(t, FMM_EINVAL, "offsets[0] must be 0");
    for (int s = 0; s < count; ++s)
        if (offsets[s + 1] < offsets[s]) return fail(t, FMM_EINVAL, "offsets must be non-decreasing");
    const int64_t n = offsets[count];
    if (n >= ((int64_t)1 << 31)) return fail(t, FMM_EINVAL, "total n out of range");
    t->sys_off.assign(offsets, offsets + count + 1);
    return set_sources_impl(t, positions, moments, n, source_order, source_order);
}

static fmm_status set_sources_impl(fmm_tree *t, const double *positions, const double *moments,
                                   int64_t n, int source_order, int source_order_hi)
{
    if (source_order < 0 || source_order > FMM_MAX_SOURCE_ORDER)
        return fail(t, FMM_EORDER, "source order must be 0, 1 or 2");
    if (n > 0 && (!positions || !moments)) return fail(t, FMM_EINVAL, "NULL positions or moments");
    DeviceGuard g(t->device);
    drop_graph(t);
    t->have_sources = false;
    t->have_lists = false;
    t->tc_plan = false;
    t->sym_plan = false;
    t->bh_ran = false;
    t->d_p = -1;
    t->n = n;
    t->s = source_order;
    t->s_hi = source_order_hi;
    t->nS = ntot(source_order_hi) - ntot(source_order - 1);
    fmm_status st = build_tree(t, positions, moments);
    if (st != FMM_OK) return st;
    if (t->profiling && n > 0) {
        FMM_TRY(cuda_check(t, cudaEventSynchronize(t->ev[3]), "event sync"));
        for (int i = 0; i < 3; ++i) cudaEventElapsedTime(&t->phase_ms[i], t->ev[i], t->ev[i + 1]);
    }
    t->have_sources = true;
    return FMM_OK;
}

fmm_status fmm_evaluate(fmm_tree *t, int p, double theta, int want_potential, int want_field,
                        double *potential, double *field)
{
    if (!t) return FMM_EINVAL;
    t->err.clear();
    if (!t->have_sources) return fail(t, FMM_ESTATE, "fmm_set_sources has not succeeded");
    if (!(theta > 0.0 && theta < 1.0)) return fail(t, FMM_EINVAL, "theta must lie in (0, 1)");
    if (!want_potential && !want_field) return fail(t, FMM_EINVAL, "nothing requested");
    if (p < 0 || p + t->s > FMM_MAX_TOTAL_ORDER || (want_field && p < 1))
        return fail(t, FMM_EORDER, "need 0 <= p, p + s <= 12, and p >= 1 for the field");
    if (t->n == 0) return FMM_OK;
    if ((want_potential && !potential) || (want_field && !field))
        return fail(t, FMM_EINVAL, "NULL output for a requested quantity");
    DeviceGuard g(t->device);
    record(t, 4);
    if (!t->have_lists || t->theta != theta) FMM_TRY(build_lists(t, theta));
    record(t, 5);
    FMM_TRY(evaluate_body(t, p, want_potential, want_field, potential, field));
    record(t, 12);
    if (t->profiling) {
        FMM_TRY(cuda_check(t, cudaEventSynchronize(t->ev[12]), "event sync"));
        for (int i = 3; i <= 10; ++i) cudaEventElapsedTime(&t->phase_ms[i], t->ev[i + 1], t->ev[i + 2]);
    }
    return FMM_OK;
}

fmm_status fmm_evaluate_bh(fmm_tree *t, int p, double theta, int want_potential, int want_field,
                           double *potential, double *field)
{
    if (!t) return FMM_EINVAL;
    t->err.clear();
    if (!t->have_sources) return fail(t, FMM_ESTATE, "fmm_set_sources has not succeeded");
    if (!(theta >= 0.0) || !std::isfinite(theta)) return fail(t, FMM_EINVAL, "theta must be finite and >= 0");
    if (!want_potential && !want_field) return fail(t, FMM_EINVAL, "nothing requested");
    if (p < t->s || p > FMM_MAX_TOTAL_ORDER)
        return fail(t, FMM_EORDER, "need s <= p <= 12 for the Barnes-Hut multipoles");
    if (t->n == 0) return FMM_OK;
    if ((want_potential && !potential) || (want_field && !field))
        return fail(t, FMM_EINVAL, "NULL output for a requested quantity");
    DeviceGuard g(t->device);
    drop_graph(t);                       // the tables a captured evaluate reads change here
    return run_bh(t, p, theta, want_potential, want_field, potential, field);
}

fmm_status fmm_get_info(const fmm_tree *t, fmm_tree_info *o)
{
    if (!t || !o) return FMM_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->n = t->n;
    o->ncells = t->ncells;
    o->nleaves = t->nleaves;
    o->nlevels = t->nlevels;
    o->source_order = t->s;
    o->source_order_hi = t->s_hi;
    o->n_m2l = t->have_lists ? t->n_m2l : 0;
    o->n_p2p = t->have_lists ? t->n_p2p : 0;
    o->n_p2p_interactions = t->have_lists ? t->n_p2p_inter : 0;
    o->n_doffsets = t->have_lists ? t->n_doff : 0;
    o->theta = t->have_lists ? t->theta : 0.0;
    o->lo[0] = t->lo[0]; o->lo[1] = t->lo[1]; o->lo[2] = t->lo[2];
    o->side = t->side;
    o->device_bytes = (int64_t)t->held;
    o->nsystems = t->sys_off.empty() ? 0 : (int64_t)t->sys_off.size() - 1;
    if (t->tc_plan && t->have_lists) {
        o->tc_tiles = t->tc_tiles;
        o->tc_rows = t->tc_rows;
        o->tc_chunks = t->tc_chunks;
    }
    if (t->bh_ran && t->b_bh_cnt.ptr) {
        unsigned long long cnt[2] = {0, 0};
        DeviceGuard g(t->device);
        if (cudaMemcpyAsync(cnt, t->b_bh_cnt.ptr, sizeof(cnt), cudaMemcpyDeviceToHost, t->stream) == cudaSuccess &&
            cudaStreamSynchronize(t->stream) == cudaSuccess) {
            o->bh_m2p = (int64_t)cnt[0];
            o->bh_p2p = (int64_t)cnt[1];
        }
    }
    return FMM_OK;
}

fmm_status fmm_copy_array(const fmm_tree *tc, fmm_array which, void *host_dst, size_t bytes,
                          size_t *written)
{
    fmm_tree *t = const_cast<fmm_tree *>(tc);
    if (!t || (!host_dst && bytes)) return FMM_EINVAL;
    DeviceGuard g(t->device);
    FMM_TRY(cuda_check(t, t->stream ? cudaStreamSynchronize(t->stream) : cudaDeviceSynchronize(),
                       "sync"));
    const int64_t n = t->n, nc = t->ncells;
    auto dl = [&](const DevBuf &b, size_t nbytes, void *dst) {
        return cuda_check(t, cudaMemcpy(dst, b.ptr, nbytes, cudaMemcpyDeviceToHost), "copy out");
    };
    auto interleave = [&](std::initializer_list<const DevBuf *> bufs, int64_t count) -> fmm_status {
        const size_t k = bufs.size(), need = 4 * k * (size_t)count;
        if (bytes < need) return fail(t, FMM_EINVAL, "buffer too small");
        std::vector<int32_t> tmp((size_t)count);
        int32_t *d = (int32_t *)host_dst;
        size_t j = 0;
        for (const DevBuf *b : bufs) {
            if (count) FMM_TRY(dl(*b, 4 * (size_t)count, tmp.data()));
            for (int64_t i = 0; i < count; ++i) d[k * i + j] = tmp[i];
            ++j;
        }
        if (written) *written = need;
        return FMM_OK;
    };
    auto plain = [&](const DevBuf &b, size_t need) -> fmm_status {
        if (bytes < need) return fail(t, FMM_EINVAL, "buffer too small");
        if (need) FMM_TRY(dl(b, need, host_dst));
        if (written) *written = need;
        return FMM_OK;
    };
    auto pairs = [&](const DevBuf &off, const DevBuf &src, int64_t np) -> fmm_status {
        if (!t->have_lists) return fail(t, FMM_ESTATE, "no interaction lists yet");
        const size_t need = 8 * (size_t)np;
        if (bytes < need) return fail(t, FMM_EINVAL, "buffer too small");
        std::vector<int32_t> o((size_t)nc + 1), s((size_t)np);
        FMM_TRY(dl(off, 4 * ((size_t)nc + 1), o.data()));
        if (np) FMM_TRY(dl(src, 4 * (size_t)np, s.data()));
        int32_t *d = (int32_t *)host_dst;
        for (int64_t c = 0; c < nc; ++c)
            for (int32_t q = o[c]; q < o[c + 1]; ++q) { d[2 * q] = (int32_t)c; d[2 * q + 1] = s[q]; }
        if (written) *written = need;
        return FMM_OK;
    };
    switch (which) {
    case FMM_ARR_KEYS: return plain(t->b_keys, 8 * (size_t)n);
    case FMM_ARR_PERM: return plain(t->b_perm, 4 * (size_t)n);
    case FMM_ARR_CELL_LEVEL: return plain(t->b_level, 4 * (size_t)nc);
    case FMM_ARR_CELL_COORD: return interleave({&t->b_cx, &t->b_cy, &t->b_cz}, nc);
    case FMM_ARR_CELL_RANGE: return interleave({&t->b_begin, &t->b_end}, nc);
    case FMM_ARR_CELL_PARENT: return plain(t->b_parent, 4 * (size_t)nc);
    case FMM_ARR_CELL_CHILD: return interleave({&t->b_child, &t->b_nchild}, nc);
    case FMM_ARR_CELL_CENTRE: return plain(t->b_centre, 24 * (size_t)nc);
    case FMM_ARR_CELL_HALF: return plain(t->b_half, 8 * (size_t)nc);
    case FMM_ARR_M2L: return pairs(t->b_m2l_off, t->b_m2l_src, t->n_m2l);
    case FMM_ARR_P2P: return pairs(t->b_p2p_off, t->b_p2p_src, t->n_p2p);
    case FMM_ARR_MULTIPOLE:
        if (t->tab_key_p < 0) return fail(t, FMM_ESTATE, "no evaluate yet");
        if (t->prec != FMM_FP64) {          // scaled FP32 rows, stored padded to 4 floats
            const int nM = t->tab.nM, ld = (nM + 3) & ~3;
            const size_t need = 4 * (size_t)nc * nM;
            if (bytes < need) return fail(t, FMM_EINVAL, "buffer too small");
            std::vector<float> pad((size_t)nc * ld);
            if (need) FMM_TRY(dl(t->b_M32, 4 * pad.size(), pad.data()));
            float *d = (float *)host_dst;
            for (int64_t c = 0; c < nc; ++c)
                std::memcpy(d + (size_t)c * nM, pad.data() + (size_t)c * ld, 4 * (size_t)nM);
            if (written) *written = need;
            return FMM_OK;
        }
        return plain(t->b_M, 8 * (size_t)nc * t->tab.nM);
    case FMM_ARR_LOCAL:
        if (t->tab_key_p < 0) return fail(t, FMM_ESTATE, "no evaluate yet");
        if (t->prec != FMM_FP64) return plain(t->b_L32, 4 * (size_t)nc * t->tab.nLh);
        return plain(t->b_L, 8 * (size_t)nc * t->tab.nLh);
    case FMM_ARR_CELL_SYSTEM: return plain(t->b_sys, 4 * (size_t)nc);
    }
    return fail(t, FMM_EINVAL, "unknown array id");
}

fmm_status fmm_direct_sum(void *cuda_stream, const double *positions, const double *moments,
                          int64_t n, int source_order, const int32_t *targets, int64_t n_targets,
                          double *potential, double *field)
{
    if (n < 0 || n_targets < 0 || source_order < 0 || source_order > FMM_MAX_SOURCE_ORDER)
        return FMM_EINVAL;
    if (n > 0 && (!positions || !moments)) return FMM_EINVAL;
    if (!targets && n_targets > n) return FMM_EINVAL;
    int64_t launches = 0;
    launch_direct((cudaStream_t)cuda_stream, positions, moments, n, source_order, source_order,
                  targets, n_targets, potential, field, &launches);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : FMM_ECUDA;
}

fmm_status fmm_direct_sum_mixed(void *cuda_stream, const double *positions, const double *moments,
                                int64_t n, int s_lo, int s_hi, const int32_t *targets,
                                int64_t n_targets, double *potential, double *field)
{
    if (n < 0 || n_targets < 0 || s_lo < 0 || s_hi < s_lo || s_hi > FMM_MAX_SOURCE_ORDER)
        return FMM_EINVAL;
    if (n > 0 && (!positions || !moments)) return FMM_EINVAL;
    if (!targets && n_targets > n) return FMM_EINVAL;
    int64_t launches = 0;
    launch_direct((cudaStream_t)cuda_stream, positions, moments, n, s_lo, s_hi, targets, n_targets,
                  potential, field, &launches);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : FMM_ECUDA;
}

fmm_status fmm_check_rsqrt(void *cuda_stream, const double *x, int64_t n, double *own,
                           double *ref)
{
    if (n < 0 || (n > 0 && (!x || !own || !ref))) return FMM_EINVAL;
    launch_check_rsqrt((cudaStream_t)cuda_stream, x, n, own, ref);
    return cudaGetLastError() == cudaSuccess ? FMM_OK : FMM_ECUDA;
}

fmm_status fmm_check_umma(const float *A, const float *B, float *D, int nkb, int N,
                          const int *kbn, int a_tmem, int passes)
{
    if (!A || !B || !D || !kbn) return FMM_EINVAL;
    unsigned *err = nullptr;
    if (cudaMalloc(&err, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return FMM_ENOMEM;
    }
    fmm_status st = FMM_OK;
    if (cudaMemset(err, 0, sizeof(unsigned)) != cudaSuccess) st = FMM_ECUDA;
    if (st == FMM_OK) st = check_umma(nullptr, A, B, D, nkb, N, kbn, a_tmem, passes, err);
    unsigned h = 0;
    if (st == FMM_OK && (cudaDeviceSynchronize() != cudaSuccess ||
                         cudaMemcpy(&h, err, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess))
        st = FMM_ECUDA;
    if (st == FMM_OK && h) st = FMM_ETIMEOUT;
    cudaFree(err);
    return st;
}

fmm_status fmm_morton_order(void *cuda_stream, const double *positions, int64_t n,
                            uint64_t *keys_out, int32_t *perm_out)
{
    if (n < 0 || n >= ((int64_t)1 << 31)) return FMM_EINVAL;
    if (n == 0) return FMM_OK;
    if (!positions || !keys_out || !perm_out) return FMM_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    void *keys2 = nullptr, *idx2 = nullptr, *hist = nullptr, *box = nullptr;
    const size_t hb = radix_hist_bytes(n);
    cudaError_t e = cudaMalloc(&keys2, 8 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&idx2, 4 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&hist, hb);
    if (e == cudaSuccess) e = cudaMalloc(&box, 256);
    fmm_status st_out = FMM_OK;
    if (e != cudaSuccess) {
        cudaGetLastError();
        st_out = FMM_ENOMEM;
    } else {
        int64_t launches = 0;
        cudaMemsetAsync((char *)box + 160, 0, 4, st);
        morton_order_raw(st, positions, n, keys_out, (uint32_t *)perm_out, (uint64_t *)keys2,
                         (uint32_t *)idx2, (uint32_t *)hist, (unsigned long long *)box, (double *)box + 8, (int *)((char *)box + 160),
                         &launches);
        int err = 0;
        e = cudaMemcpyAsync(&err, (char *)box + 160, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) st_out = FMM_ECUDA;
        else if (err & kErrNonFinite) st_out = FMM_EINVAL;
        else if (err & kErrSortWait) st_out = FMM_ETIMEOUT;
    }
    cudaFree(keys2); cudaFree(idx2); cudaFree(hist); cudaFree(box);
    return st_out;
}

}  // extern "C"
