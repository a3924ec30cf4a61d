// graph.cu -- repeated evaluation of one geometry: moment updates, the
// evaluate captured as a CUDA graph, and the autotuner that picks the
// handle's kernel variants by timing them on its own workload.
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

struct Guard {
    int prev = -1;
    explicit Guard(int d)
    {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~Guard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// S[k] = moments[perm[k]]: the caller's order into the tree's sorted order
__global__ void k_gather_moments(const double *mom, int nS, const int32_t *perm, int64_t n, double *S)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t o = perm[k];
    for (int a = 0; a < nS; ++a) S[k * nS + a] = mom[o * nS + a];
}

fmm_status fail(fmm_tree *t, fmm_status s, const char *msg)
{
    t->err = msg;
    return s;
}

}  // namespace

void drop_graph(fmm_tree *t)
{
    if (t->graph_exec) cudaGraphExecDestroy(t->graph_exec);
    if (t->graph) cudaGraphDestroy(t->graph);
    t->graph_exec = nullptr;
    t->graph = nullptr;
    t->g_p = -1;
}

}  // namespace fmm

using namespace fmm;

fmm_status fmm_update_moments(fmm_tree *t, const double *moments)
{
    if (!t) return FMM_EINVAL;
    t->err.clear();
    if (!t->have_sources) return fail(t, FMM_ESTATE, "fmm_set_sources has not succeeded");
    if (t->n == 0) return FMM_OK;
    if (!moments) return fail(t, FMM_EINVAL, "NULL moments");
    Guard g(t->device);
    k_gather_moments<<<(unsigned)((t->n + 255) / 256), 256, 0, t->stream>>>(
        moments, t->nS, (const int32_t *)t->b_perm.ptr, t->n, (double *)t->b_S.ptr);
    ++t->launches;
    return cuda_check(t, cudaGetLastError(), "moment gather");
}

fmm_status fmm_evaluate_graph(fmm_tree *t, int p, double theta, int want_potential, int want_field,
                              double *potential, double *field)
{
    if (!t) return FMM_EINVAL;
    const bool same = t->graph_exec && t->g_p == p && t->g_theta == theta && t->g_phi == want_potential &&
                      t->g_field == want_field && t->g_pot == potential && t->g_fld == field;
    Guard g(t->device);
    if (same) {
        t->err.clear();
        FMM_TRY(cuda_check(t, cudaGraphLaunch(t->graph_exec, t->stream), "graph launch"));
        t->launches += 1;
        return FMM_OK;
    }
    // an ordinary evaluate first: it validates the arguments and brings every
    // cache (lists, tables, D rows, plan, operator images, buffers) up to date,
    // so that the captured evaluate makes no allocation and no host sync
    FMM_TRY(fmm_evaluate(t, p, theta, want_potential, want_field, potential, field));
    if (t->n == 0) return FMM_OK;
    drop_graph(t);
    if (!t->cap_stream)
        FMM_TRY(cuda_check(t, cudaStreamCreateWithFlags(&t->cap_stream, cudaStreamNonBlocking), "stream"));
    FMM_TRY(cuda_check(t, cudaStreamSynchronize(t->stream ? t->stream : (cudaStream_t)0), "sync"));
    cudaStream_t user = t->stream;
    const bool prof = t->profiling;
    const int64_t launches = t->launches;
    t->stream = t->cap_stream;
    t->profiling = false;
    fmm_status st = cuda_check(t, cudaStreamBeginCapture(t->cap_stream, cudaStreamCaptureModeThreadLocal),
                               "begin capture");
    if (st == FMM_OK) {
        st = evaluate_body(t, p, want_potential, want_field, potential, field);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(t->cap_stream, &graph);
        if (st == FMM_OK) st = cuda_check(t, e, "end capture");
        if (st == FMM_OK) {
            t->graph = graph;
            st = cuda_check(t, cudaGraphInstantiate(&t->graph_exec, graph, 0), "graph instantiate");
        } else if (graph) {
            cudaGraphDestroy(graph);
        }
    }
    t->stream = user;
    t->profiling = prof;
    t->launches = launches;
    if (st != FMM_OK) {
        cudaGetLastError();
        drop_graph(t);
        return st;
    }
    t->g_p = p;
    t->g_theta = theta;
    t->g_phi = want_potential;
    t->g_field = want_field;
    t->g_pot = potential;
    t->g_fld = field;
    return FMM_OK;
}

fmm_status fmm_autotune(fmm_tree *t, int p, double theta, int want_potential, int want_field,
                        double *potential, double *field, int reps, fmm_tuning *out)
{
    if (!t) return FMM_EINVAL;
    if (reps < 1 || reps > 1000) return fail(t, FMM_EINVAL, "reps must be in [1, 1000]");
    // candidates: variants that compute the same sums in another order (the
    // three FP64 P2P kernels agree to FP64 rounding; the M2L paths of FMM_3XTF32
    // and its chunk lengths agree to FP32 rounding).  The FP32 forms keep their
    // P2P kernel: only the one-way kernel evaluates the close pairs in
    // double-float, so the symmetric one would trade accuracy for time.
    std::vector<fmm_tuning> cand;
    fmm_tuning base;
    std::memset(&base, 0, sizeof(base));
    base.p2p_variant = t->p2p_variant;
    base.m2l_tensor = t->m2l_simt ? 0 : 1;
    base.tc_chunk_rows = t->tc_G > 0 ? t->tc_G : 16;
    base.m2l_harmonic = t->m2l_harmonic ? 1 : 0;
    base.p2p_targets = t->p2p_tt;
    base.m2l_tiled = t->m2l_tiled ? 1 : 0;
    if (t->prec == FMM_FP64) {
        for (int v : {0, 1, 2}) {
            fmm_tuning c = base;
            c.p2p_variant = v;
            cand.push_back(c);
        }
    } else if (t->prec == FMM_3XTF32) {
        for (int G : {8, 16, 32}) {
            fmm_tuning c = base;
            c.m2l_tensor = 1;
            c.tc_chunk_rows = G;
            cand.push_back(c);
        }
        fmm_tuning c = base;
        c.m2l_tensor = 0;
        c.m2l_tiled = 1;
        cand.push_back(c);
    } else {
        for (int G : {8, 16, 32}) {
            fmm_tuning c = base;
            c.m2l_tiled = 1;
            c.tc_chunk_rows = G;
            cand.push_back(c);
        }
        fmm_tuning c = base;
        c.m2l_tiled = 0;
        cand.push_back(c);
    }
    // the FP32 forms' second stage: the winner with the other P2P tile shape
    const size_t stage1 = cand.size();
    Guard g(t->device);
    drop_graph(t);
    cudaEvent_t a = nullptr, b = nullptr;
    FMM_TRY(cuda_check(t, cudaEventCreate(&a), "event"));
    FMM_TRY(cuda_check(t, cudaEventCreate(&b), "event"));
    fmm_status st = FMM_OK;
    int best = -1;
    float best_ms = std::numeric_limits<float>::infinity();
    for (size_t k = 0; k < cand.size() && st == FMM_OK; ++k) {
        const fmm_tuning c = cand[k];
        t->p2p_variant = c.p2p_variant;
        t->p2p_tt = c.p2p_targets;
        t->m2l_simt = !c.m2l_tensor;
        t->m2l_tiled = c.m2l_tiled != 0;
        if (t->tc_G != c.tc_chunk_rows) {
            t->tc_G = c.tc_chunk_rows;
            t->tc_plan = false;
        }
        st = fmm_evaluate(t, p, theta, want_potential, want_field, potential, field);   // warm
        if (st != FMM_OK) break;
        cudaEventRecord(a, t->stream);
        for (int r = 0; r < reps && st == FMM_OK; ++r)
            st = fmm_evaluate(t, p, theta, want_potential, want_field, potential, field);
        cudaEventRecord(b, t->stream);
        if (st != FMM_OK) break;
        st = cuda_check(t, cudaEventSynchronize(b), "event sync");
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        cand[k].ms_per_evaluate = ms / reps;
        if (ms < best_ms) {
            best_ms = ms;
            best = (int)k;
        }
        if (k + 1 == stage1 && t->prec != FMM_FP64) {
            fmm_tuning c2 = cand[best];
            c2.p2p_targets = c2.p2p_targets == 1 ? 2 : 1;
            cand.push_back(c2);
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != FMM_OK) return st;
    const fmm_tuning &c = cand[best];
    t->p2p_variant = c.p2p_variant;
    t->p2p_tt = c.p2p_targets;
    t->m2l_simt = !c.m2l_tensor;
    t->m2l_tiled = c.m2l_tiled != 0;
    if (t->tc_G != c.tc_chunk_rows) {
        t->tc_G = c.tc_chunk_rows;
        t->tc_plan = false;
    }
    t->tuned = true;
    if (out) {
        *out = c;
        out->candidates = (int)cand.size();
    }
    return FMM_OK;
}

fmm_status fmm_set_tuning(fmm_tree *t, const fmm_tuning *tuning)
{
    if (!t) return FMM_EINVAL;
    t->err.clear();
    if (!tuning) return fail(t, FMM_EINVAL, "NULL tuning");
    const fmm_tuning &c = *tuning;
    if (c.p2p_variant > 2) return fail(t, FMM_EINVAL, "p2p_variant must be 0, 1 or 2");
    if (c.m2l_tensor > 1) return fail(t, FMM_EINVAL, "m2l_tensor must be 0 or 1");
    if (c.tc_chunk_rows == 0 || c.tc_chunk_rows > 64)
        return fail(t, FMM_EINVAL, "tc_chunk_rows must be in [1, 64]");
    if (c.m2l_harmonic > 1) return fail(t, FMM_EINVAL, "m2l_harmonic must be 0 or 1");
    if (c.p2p_targets > 2) return fail(t, FMM_EINVAL, "p2p_targets must be 1 or 2");
    if (c.m2l_tiled > 1) return fail(t, FMM_EINVAL, "m2l_tiled must be 0 or 1");
    drop_graph(t);
    if (c.p2p_variant >= 0) t->p2p_variant = c.p2p_variant;
    if (c.m2l_tensor >= 0) t->m2l_simt = c.m2l_tensor == 0;
    if (c.m2l_harmonic >= 0) t->m2l_harmonic = c.m2l_harmonic == 1;
    if (c.p2p_targets > 0) t->p2p_tt = c.p2p_targets;
    if (c.m2l_tiled >= 0) t->m2l_tiled = c.m2l_tiled == 1;
    if (c.tc_chunk_rows > 0 && t->tc_G != c.tc_chunk_rows) {
        t->tc_G = c.tc_chunk_rows;
        t->tc_plan = false;
    }
    return FMM_OK;
}
