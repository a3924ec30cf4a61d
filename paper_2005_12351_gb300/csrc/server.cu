// server.cu -- continuous-batching request server over the FMM handles.
//
// A server owns `slots` workers.  Each worker has its own CUDA stream and a
// long-lived fmm_tree handle whose device buffers stay resident between
// requests, so a request's tree, lists and expansions live on the device for
// as long as it runs and the next request on that slot reuses the memory.
// Requests are admitted in arrival order as soon as (a) a slot is idle and
// (b) the request's estimated device memory fits the server's budget next to
// what the other slots hold; requests admitted while others run overlap on
// the GPU through the separate streams.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "fmm_internal.cuh"

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Upper estimate of a request's device memory (bytes): particle arrays
// (keys, indices, sorted copies, outputs, FP32 copies), cells with their M
// and L rows, the interaction lists and their sort scratch.
size_t estimate_bytes(int64_t n, int s, int p, int max_leaf)
{
    const int nS = (s + 1) * (s + 2) / 2;
    const int64_t nM = fmm::ntot(p + s) - fmm::ntot(s - 1), nL = fmm::ntot(p);
    const int64_t cells = 4 * (n / std::max(1, max_leaf)) + 64;
    const int64_t m2l = 320 * cells, p2p = 40 * cells;
    size_t b = 0;
    b += (size_t)n * (8 * 2 + 4 * 2 + 24 + 8 * nS + 4 + 8 + 24 + 32 + 4 * (nS + 1));
    b += (size_t)cells * (4 * 12 + 32 + 8 * (nM + nL) + 4 * (nM + nL) + 8 * 8);
    b += (size_t)m2l * (8 + 8 + 8 + 4 + 4 + 4) + (size_t)p2p * (8 + 8 + 8 + 4 + 4);
    b += (size_t)fmm::ntot(p + s) * 8 * 4096;
    // list build scratch (hash table, frontier growth, sort ping-pong) is not
    // tracked term by term: double the sum and add a fixed allowance
    return 2 * b + (64u << 20);
}

struct Job {
    int64_t ticket;
    fmm_request req;
    fmm_request_result res;
    size_t est;
    bool done = false;
};

}  // namespace

struct fmm_server {
    int device = 0;
    fmm_precision prec = FMM_FP64;
    size_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> queue;
    std::map<int64_t, Job *> jobs;
    int64_t next_ticket = 1;
    bool stopping = false;
    struct Slot {
        std::thread th;
        cudaStream_t stream = nullptr;
        fmm_tree *tree = nullptr;
        Job *job = nullptr;
        size_t held = 0;        // device bytes the slot's handle holds
        size_t reserved = 0;    // estimate of the running job
    };
    std::vector<Slot> slots;
    int64_t completed = 0, failed = 0;
    size_t peak_bytes = 0;
    double first_start = 0.0, last_end = 0.0;
    int64_t particles_done = 0;

    // device memory promised to the slots: what idle slots hold, and for a
    // running slot what it held when the job started plus the job's estimate
    // (a handle's buffers only grow, so a job may add its estimate on top)
    size_t committed_locked(const Slot *except) const
    {
        size_t c = 0;
        for (const Slot &s : slots)
            if (&s != except) c += s.held + s.reserved;
        return c;
    }
};

namespace {

void run_job(fmm_server *sv, fmm_server::Slot &sl, Job *j)
{
    const fmm_request &r = j->req;
    fmm_tree *t = sl.tree;
    fmm_status st = FMM_OK;
    double *d_pos = nullptr, *d_mom = nullptr, *d_phi = nullptr, *d_E = nullptr;
    const int nS = (r.source_order + 1) * (r.source_order + 2) / 2;
    cudaSetDevice(sv->device);
    if (t->max_leaf != r.max_leaf) t->max_leaf = r.max_leaf;
    // inputs and outputs through the handle's own grow-only staging buffers
    const size_t bp = 24 * (size_t)r.n, bm = 8 * (size_t)r.n * nS;
    st = fmm::ensure(t, t->b_req_in, std::max<size_t>(bp + bm, 16));
    if (st == FMM_OK) st = fmm::ensure(t, t->b_req_out, std::max<size_t>(32 * (size_t)r.n, 16));
    if (st == FMM_OK && r.n > 0) {
        d_pos = (double *)t->b_req_in.ptr;
        d_mom = (double *)((char *)t->b_req_in.ptr + bp);
        d_phi = (double *)t->b_req_out.ptr;
        d_E = d_phi + r.n;
        cudaMemcpyAsync(d_pos, r.positions, bp, cudaMemcpyHostToDevice, sl.stream);
        cudaMemcpyAsync(d_mom, r.moments, bm, cudaMemcpyHostToDevice, sl.stream);
    }
    if (st == FMM_OK) st = fmm_set_sources(t, d_pos, d_mom, r.n, r.source_order);
    if (st == FMM_OK)
        st = fmm_evaluate(t, r.p, r.theta, r.want_potential, r.want_field,
                          r.want_potential ? d_phi : nullptr, r.want_field ? d_E : nullptr);
    if (st == FMM_OK && r.n > 0) {
        if (r.want_potential && r.potential)
            cudaMemcpyAsync(r.potential, d_phi, 8 * (size_t)r.n, cudaMemcpyDeviceToHost, sl.stream);
        if (r.want_field && r.field)
            cudaMemcpyAsync(r.field, d_E, 24 * (size_t)r.n, cudaMemcpyDeviceToHost, sl.stream);
    }
    cudaError_t e = cudaStreamSynchronize(sl.stream);
    if (st == FMM_OK && e != cudaSuccess) st = FMM_ECUDA;
    fmm_tree_info inf;
    fmm_get_info(t, &inf);
    j->res.status = st;
    j->res.end_s = now_s();
    j->res.device_bytes = inf.device_bytes;
    std::strncpy(j->res.message, fmm_last_error(t), sizeof(j->res.message) - 1);
}

// Release the device buffers of idle workers (their handles are not in use).
void trim_idle_locked(fmm_server *sv)
{
    for (auto &s : sv->slots) {
        if (s.job || s.held == 0 || !s.tree) continue;
        fmm_tree *nt = nullptr;
        if (fmm_create_tree(&nt, sv->device, s.stream, 64, sv->prec, 0) != FMM_OK) continue;
        fmm_destroy(s.tree);
        s.tree = nt;
        fmm_tree_info inf;
        fmm_get_info(s.tree, &inf);
        s.held = (size_t)inf.device_bytes;
    }
}

void worker(fmm_server *sv, int idx)
{
    fmm_server::Slot &sl = sv->slots[idx];
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        // admission: the head of the queue runs here once its estimate fits
        sv->cv_work.wait(lk, [&] {
            if (sv->stopping && sv->queue.empty()) return true;
            if (sv->queue.empty()) return false;
            const Job *h = sv->queue.front();
            if (sv->committed_locked(&sl) + sl.held + h->est <= sv->budget) return true;
            bool any_running = false;
            for (const auto &s : sv->slots) any_running |= s.job != nullptr;
            if (!any_running) {           // only idle memory stands in the way
                trim_idle_locked(sv);
                return sv->committed_locked(&sl) + sl.held + h->est <= sv->budget;
            }
            return false;
        });
        if (sv->queue.empty()) break;
        Job *j = sv->queue.front();
        sv->queue.pop_front();
        sl.job = j;
        sl.reserved = j->est;
        j->res.slot = idx;
        j->res.start_s = now_s();
        if (sv->first_start == 0.0) sv->first_start = j->res.start_s;
        // the handle may grow to what was admitted for it, never further
        sl.tree->budget = sv->budget == (size_t)-1 ? 0 : sl.held + j->est;
        lk.unlock();
        run_job(sv, sl, j);
        lk.lock();
        fmm_tree_info inf;
        fmm_get_info(sl.tree, &inf);
        sl.held = (size_t)inf.device_bytes;
        sl.reserved = 0;
        sl.job = nullptr;
        j->done = true;
        if (j->res.status == FMM_OK) {
            ++sv->completed;
            sv->particles_done += j->req.n;
        } else {
            ++sv->failed;
        }
        sv->last_end = std::max(sv->last_end, j->res.end_s);
        sv->peak_bytes = std::max(sv->peak_bytes, sv->committed_locked(nullptr));
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

fmm_status fmm_server_create(fmm_server **out, int device, int slots, fmm_precision prec,
                             size_t mem_budget_bytes)
{
    if (!out || slots < 1 || slots > 64) return FMM_EINVAL;
    *out = nullptr;
    fmm_server *sv = new (std::nothrow) fmm_server();
    if (!sv) return FMM_ENOMEM;
    sv->device = device;
    sv->prec = prec;
    sv->budget = mem_budget_bytes ? mem_budget_bytes : (size_t)-1;
    sv->slots.resize(slots);
    for (int i = 0; i < slots; ++i) {
        fmm_server::Slot &sl = sv->slots[i];
        cudaSetDevice(device);
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            fmm_server_destroy(sv);
            return FMM_ECUDA;
        }
        fmm_status st = fmm_create_tree(&sl.tree, device, sl.stream, 64, prec, 0);
        if (st != FMM_OK) {
            fmm_server_destroy(sv);
            return st;
        }
        fmm_tree_info inf;
        fmm_get_info(sl.tree, &inf);
        sl.held = (size_t)inf.device_bytes;
    }
    for (int i = 0; i < slots; ++i) sv->slots[i].th = std::thread(worker, sv, i);
    *out = sv;
    return FMM_OK;
}

fmm_status fmm_server_submit(fmm_server *sv, const fmm_request *r, int64_t *ticket)
{
    if (!sv || !r || !ticket) return FMM_EINVAL;
    if (r->n < 0 || r->source_order < 0 || r->source_order > FMM_MAX_SOURCE_ORDER ||
        r->p < 0 || r->p + r->source_order > FMM_MAX_TOTAL_ORDER || r->max_leaf < 1 ||
        !(r->theta > 0.0 && r->theta < 1.0) || (r->n > 0 && (!r->positions || !r->moments)))
        return FMM_EINVAL;
    Job *j = new (std::nothrow) Job();
    if (!j) return FMM_ENOMEM;
    j->req = *r;
    std::memset(&j->res, 0, sizeof(j->res));
    j->res.submit_s = now_s();
    j->est = estimate_bytes(r->n, r->source_order, r->p, r->max_leaf);
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stopping) { delete j; return FMM_ESTATE; }
    if (j->est + (64u << 20) > sv->budget) { delete j; return FMM_EBUDGET; }   // could never fit
    j->ticket = sv->next_ticket++;
    j->res.ticket = j->ticket;
    sv->jobs[j->ticket] = j;
    sv->queue.push_back(j);
    *ticket = j->ticket;
    sv->cv_work.notify_all();
    return FMM_OK;
}

fmm_status fmm_server_poll(fmm_server *sv, int64_t ticket, int *done)
{
    if (!sv || !done) return FMM_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return FMM_EINVAL;
    *done = it->second->done ? 1 : 0;
    return FMM_OK;
}

fmm_status fmm_server_wait(fmm_server *sv, int64_t ticket, fmm_request_result *res)
{
    if (!sv) return FMM_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return FMM_EINVAL;
    Job *j = it->second;
    sv->cv_done.wait(lk, [&] { return j->done; });
    if (res) *res = j->res;
    sv->jobs.erase(it);
    fmm_status st = j->res.status;
    delete j;
    return st;
}

fmm_status fmm_server_get_stats(fmm_server *sv, fmm_server_stats *out)
{
    if (!sv || !out) return FMM_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    std::memset(out, 0, sizeof(*out));
    out->completed = sv->completed;
    out->failed = sv->failed;
    out->queued = (int64_t)sv->queue.size();
    int running = 0;
    for (const auto &s : sv->slots) running += s.job != nullptr;
    out->running = running;
    out->device_bytes = (int64_t)sv->committed_locked(nullptr);
    out->peak_device_bytes = (int64_t)sv->peak_bytes;
    out->particles_done = sv->particles_done;
    out->busy_span_s = sv->last_end > sv->first_start ? sv->last_end - sv->first_start : 0.0;
    return FMM_OK;
}

fmm_status fmm_server_destroy(fmm_server *sv)
{
    if (!sv) return FMM_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
        sv->cv_work.notify_all();
    }
    for (auto &s : sv->slots)
        if (s.th.joinable()) s.th.join();
    for (auto &s : sv->slots) {
        if (s.tree) fmm_destroy(s.tree);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    for (auto &kv : sv->jobs) delete kv.second;
    delete sv;
    return FMM_OK;
}

}  // extern "C"
