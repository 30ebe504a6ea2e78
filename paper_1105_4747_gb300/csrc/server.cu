// server.cu -- the serving loop (lya_server_*): a worker thread that admits
// extraction requests by memory budget and runs them in steps, each step one
// launch of a captured CUDA graph (the persistent optical-depth kernel, then
// the batched mean-flux root-find).  The admission and packing rules live in
// serve_sched.h; this file owns the device buffers, the graph, the worker and
// the C ABI.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lya.h"
#include "lya_internal.h"
#include "serve_internal.h"
#include "serve_sched.h"

namespace {

using lya::TauLaunch;
using namespace lya::serve;

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

constexpr size_t align16(size_t x) { return (x + 15) / 16 * 16; }
constexpr int64_t kMaxItems = 1 << 15;
constexpr int64_t kMaxUnits = 1 << 15;
constexpr int kClasses = 14;                 // skewer-length classes: n_pix in (2^(k-1), 2^k]

int length_class(int n_pix)
{
    int k = 0;
    while ((1 << k) < n_pix && k < kClasses - 1) ++k;
    return k;
}

// Threads per skewer of the standalone kernel, as a group shift of a
// 1024-thread CTA: the starting point before any tuning.
int default_shift(int n_pix)
{
    const int threads = n_pix >= 2048 ? 512 : (n_pix >= 512 ? 256 : 128);
    int s = 0;
    while ((kTauThreads >> s) > threads && s < kMaxShift) ++s;
    return s;
}

// Estimated optical-depth cost of one pixel (ns at full GPU) for a request
// with ppx sources per pixel: a fixed part (loads, sort, envelopes) and a
// per-pair part.  Only its ratios matter: it sets the step quota's packing.
double model_ns_per_px(double ppx) { return 0.012 + 0.0013 * ppx; }

struct ReqHost {
    lya_field field = nullptr;
    TauLaunch L{};
    std::vector<int64_t> ids;
    double Ft = 0.8;
    lya_server_result res{};
};

}  // namespace

struct lya_server_s {
    lya_server_config cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t dyn_smem = 0;
    int n_sm = 1;
    int rf_grid = 1;
    int kernels_per_step = 0;

    unsigned char* d_arena = nullptr;
    unsigned char* d_step = nullptr;
    unsigned char* h_step = nullptr;
    size_t step_cap = 0;
    void* d_states = nullptr;
    SlotResult* d_results = nullptr;       // max_slots results, then the error word
    SlotResult* h_results = nullptr;
    size_t results_bytes = 0;
    void* d_part = nullptr;
    void* d_spart = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    Scheduler* sched = nullptr;
    std::unordered_map<uint64_t, ReqHost> reqs;
    std::vector<uint64_t> slot_ticket;
    uint64_t next_ticket = 1;
    bool stop = false;
    bool tuning = false;
    lya_status failed = LYA_OK;
    std::thread worker;

    uint64_t steps = 0, submitted = 0, completed = 0, n_failed = 0;
    int tuned_shift[kClasses];
    double cost_scale[kClasses];
};

namespace {

lya_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return LYA_OK;
    if (e == cudaErrorMemoryAllocation) return LYA_ENOMEM;
    return LYA_ECUDA;
}

int* err_word(lya_server s) { return reinterpret_cast<int*>(s->d_results + s->cfg.max_slots); }
int host_err_word(lya_server s) { return *reinterpret_cast<int*>(s->h_results + s->cfg.max_slots); }

// Largest shift (skewers per CTA) that fits the skewer length and the
// shared memory, starting from the tuned or default choice.
int fit_shift(lya_server s, int n_pix, int w_max, int want)
{
    int sh = std::min(std::max(want, 0), kMaxShift);
    while (sh > 0 && (n_pix > kTauMaxQ * (kTauThreads >> sh) ||
                      (serve_group_smem(n_pix, w_max) << sh) > s->dyn_smem))
        --sh;
    if (n_pix > kTauMaxQ * (kTauThreads >> sh) || serve_group_smem(n_pix, w_max) > s->dyn_smem) return -1;
    return sh;
}

double sources_per_pixel(const TauLaunch& L, const lya_field f)
{
    const double T = L.t_mode ? L.T0_d : std::max((double)f->temp_max * 0.5, 1e3);
    // nsigma b(T)/du = h_coef / (c_coef sqrt(1e4/T) du)
    return 1.0 + 2.0 * L.h_coef_d / (L.c_coef_d * std::sqrt(1e4 / T) * L.du_d);
}

// Lays out one step's tables in the pinned buffer; returns the bytes used.
size_t build_step(lya_server s, const StepPlan& p)
{
    unsigned char* b = s->h_step;
    StepHeader* h = reinterpret_cast<StepHeader*>(b);
    std::memset(h, 0, sizeof(StepHeader));
    size_t off = align16(sizeof(StepHeader));
    h->off_slots = off;
    std::vector<int> local(s->cfg.max_slots, -1);
    TauLaunch* Ls = reinterpret_cast<TauLaunch*>(b + off);
    for (size_t k = 0; k < p.tau_slots.size(); ++k) {
        const int slot = p.tau_slots[k];
        local[slot] = (int)k;
        Ls[k] = s->reqs.at(s->slot_ticket[slot]).L;
    }
    h->n_slots = (int)p.tau_slots.size();
    off = align16(off + sizeof(TauLaunch) * p.tau_slots.size());
    h->off_tasks = off;
    TauTask* T = reinterpret_cast<TauTask*>(b + off);
    for (size_t k = 0; k < p.tasks.size(); ++k)
        T[k] = TauTask{local[p.tasks[k].slot], p.tasks[k].first_item, p.tasks[k].n_items, p.tasks[k].shift};
    h->n_tasks = (int)p.tasks.size();
    off = align16(off + sizeof(TauTask) * p.tasks.size());
    h->off_items = off;
    TauItem* I = reinterpret_cast<TauItem*>(b + off);
    for (size_t k = 0; k < p.items.size(); ++k) {
        const ReqHost& r = s->reqs.at(s->slot_ticket[p.items[k].slot]);
        I[k] = TauItem{(long long)r.ids[(size_t)p.items[k].row], (long long)p.items[k].row};
    }
    h->n_items = (int)p.items.size();
    off = align16(off + sizeof(TauItem) * p.items.size());
    h->off_rf = off;
    RfSlot* R = reinterpret_cast<RfSlot*>(b + off);
    for (size_t k = 0; k < p.rf.size(); ++k) {
        const StepPlan::Rf& f = p.rf[k];
        const uint64_t t = s->slot_ticket[f.slot];
        const Request* q = s->sched->find(t);
        const ReqHost& r = s->reqs.at(t);
        RfSlot x{};
        x.tau = reinterpret_cast<const float*>(s->d_arena + q->tau_off);
        x.flux = reinterpret_cast<float*>(s->d_arena + q->flux_off);
        x.n = q->pixels();
        x.Ft = r.Ft;
        x.tol = s->cfg.tol;
        x.state = f.slot;
        x.init = f.init;
        x.unit_first = f.unit_first;
        x.unit_count = f.unit_count;
        x.max_iter = s->cfg.max_iter;
        R[k] = x;
    }
    h->n_rf = (int)p.rf.size();
    off = align16(off + sizeof(RfSlot) * p.rf.size());
    h->off_units = off;
    RfUnit* U = reinterpret_cast<RfUnit*>(b + off);
    for (size_t k = 0; k < p.units.size(); ++k) U[k] = RfUnit{p.units[k].rf, 0, p.units[k].begin, p.units[k].end};
    h->n_units = (int)p.units.size();
    off = align16(off + sizeof(RfUnit) * p.units.size());
    return off;
}

size_t step_capacity(int max_slots)
{
    return align16(sizeof(StepHeader)) + align16(sizeof(TauLaunch) * max_slots) + align16(sizeof(TauTask) * kMaxItems) +
           align16(sizeof(TauItem) * kMaxItems) + align16(sizeof(RfSlot) * max_slots) +
           align16(sizeof(RfUnit) * kMaxUnits);
}

// Fill a finished request's public result from the slot's device result.
void complete(lya_server s, uint64_t ticket, const SlotResult& r)
{
    ReqHost& q = s->reqs.at(ticket);
    const Request* sq = s->sched->find(ticket);
    q.res.done = 1;
    q.res.status = (lya_status)r.status;
    q.res.A = r.A;
    q.res.iterations = r.iter;
    q.res.t_done_ns = now_ns();
    if (r.status == LYA_OK) {
        const double nn = (double)sq->pixels();
        const double m1 = r.m1 / nn, m2 = r.m2 / nn;
        q.res.stats.mean_flux = 0.5 + m1;
        q.res.stats.var_flux = m2 - m1 * m1;
        q.res.stats.tau_eff = -std::log(q.res.stats.mean_flux);
        for (int k = 0; k < 21; ++k) q.res.stats.pdf[k] = (int64_t)r.pdf[k];
        q.res.stats.n = sq->pixels();
        q.res.flux = reinterpret_cast<const float*>(s->d_arena + sq->flux_off);
        ++s->completed;
    } else {
        q.res.flux = nullptr;
        ++s->n_failed;
    }
    q.field->users.fetch_sub(1);
    s->sched->finish(ticket);
}

void fail_request(lya_server s, uint64_t ticket, lya_status why)
{
    ReqHost& q = s->reqs.at(ticket);
    if (q.res.done) return;
    q.res.done = 1;
    q.res.status = why;
    q.res.flux = nullptr;
    q.res.t_done_ns = now_ns();
    q.field->users.fetch_sub(1);
    ++s->n_failed;
    s->sched->fail(ticket);
}

void fail_all(lya_server s, lya_status why)
{
    std::vector<uint64_t> open;
    for (auto& kv : s->reqs)
        if (!kv.second.res.done) open.push_back(kv.first);
    for (uint64_t t : open) fail_request(s, t, why);
}

void worker_main(lya_server s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_work.wait(lk, [&] { return s->stop || (!s->tuning && s->sched->has_work()); });
        if (s->stop) break;
        const uint64_t t_admit = now_ns();
        for (uint64_t t : s->sched->admit()) {
            const Request* q = s->sched->find(t);
            ReqHost& r = s->reqs.at(t);
            s->slot_ticket[q->slot] = t;
            r.L.tau_out = reinterpret_cast<float*>(s->d_arena + q->tau_off);
            r.res.t_admit_ns = t_admit;
        }
        const StepPlan plan = s->sched->plan();
        if (plan.empty()) {
            // nothing runnable: the queue head waits for memory that a
            // release (which notifies) will free
            s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
            continue;
        }
        const size_t bytes = build_step(s, plan);
        lk.unlock();
        cudaError_t e = cudaMemcpyAsync(s->d_step, s->h_step, bytes, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(s->graph_exec, s->stream);
        if (e == cudaSuccess) lya::count_launch(s->kernels_per_step);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->h_results, s->d_results, s->results_bytes, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        lk.lock();
        ++s->steps;
        if (e != cudaSuccess) {
            s->failed = LYA_ECUDA;
            fail_all(s, LYA_ECUDA);
            s->cv_done.notify_all();
            break;
        }
        if (host_err_word(s) != 0) {
            // a skewer id or a field row changed under the kernel: fail this step's extractions
            for (int slot : plan.tau_slots) fail_request(s, s->slot_ticket[slot], LYA_EINVAL);
            const int zero = 0;
            cudaMemcpy(err_word(s), &zero, sizeof(int), cudaMemcpyHostToDevice);
        }
        for (const StepPlan::Rf& f : plan.rf) {
            const uint64_t t = s->slot_ticket[f.slot];
            const Request* q = s->sched->find(t);
            if (!q || q->phase == Phase::kDone) continue;
            const SlotResult& r = s->h_results[f.slot];
            if (r.final) complete(s, t, r);
        }
        s->cv_done.notify_all();
    }
}

void destroy_buffers(lya_server s)
{
    if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    cudaFree(s->d_arena);
    cudaFree(s->d_step);
    cudaFree(s->d_states);
    cudaFree(s->d_results);
    cudaFree(s->d_part);
    cudaFree(s->d_spart);
    cudaFreeHost(s->h_step);
    cudaFreeHost(s->h_results);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s->sched;
}

bool fill_result(lya_server s, uint64_t ticket, lya_server_result* out)
{
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return false;
    if (out) *out = it->second.res;
    return true;
}

}  // namespace

extern "C" {

lya_status lya_server_create(const lya_server_config* cfg, lya_server* out)
{
    if (!out) return LYA_EINVAL;
    *out = nullptr;
    if (!cfg || cfg->hbm_budget_bytes < ((size_t)1 << 20) || cfg->max_slots < 1 || cfg->max_slots > 4096 ||
        !(cfg->step_target_us > 0.0) || !(cfg->tol > 0.0) || cfg->max_iter < 1)
        return LYA_EINVAL;
    lya_server s = new (std::nothrow) lya_server_s();
    if (!s) return LYA_ENOMEM;
    s->cfg = *cfg;
    for (int k = 0; k < kClasses; ++k) {
        s->tuned_shift[k] = -1;
        s->cost_scale[k] = 1.0;
    }
    cudaGetDevice(&s->device);
    s->n_sm = lya::sm_count();
    s->rf_grid = 4 * s->n_sm;
    Limits lim;
    lim.budget = cfg->hbm_budget_bytes;
    lim.max_slots = cfg->max_slots;
    lim.step_quota_ns = cfg->step_target_us * 1e3;
    lim.max_items = kMaxItems;
    lim.max_units = kMaxUnits;
    s->sched = new (std::nothrow) Scheduler(lim);
    if (!s->sched) {
        delete s;
        return LYA_ENOMEM;
    }
    s->slot_ticket.assign(cfg->max_slots, 0);
    s->step_cap = step_capacity(cfg->max_slots);
    s->results_bytes = sizeof(SlotResult) * cfg->max_slots + 16;
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_arena, s->sched->arena().capacity());
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_step, s->step_cap);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s->h_step, s->step_cap);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_states, serve_state_bytes() * cfg->max_slots);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_results, s->results_bytes);
    if (e == cudaSuccess) e = cudaMemset(s->d_results, 0, s->results_bytes);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s->h_results, s->results_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_part, serve_part_bytes() * kMaxUnits);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_spart, serve_spart_bytes() * kMaxUnits);
    if (e == cudaSuccess) e = serve_tau_prepare(&s->dyn_smem);
    if (e == cudaSuccess) {
        // the graph of one step: every kernel reads the step buffer, so the
        // same graph serves every step
        e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t el = serve_tau_launch(s->d_step, s->dyn_smem, s->n_sm, s->stream);
            int n_rf = 0;
            if (el == cudaSuccess)
                el = serve_rf_launch(s->d_step, s->d_states, s->d_results, s->d_part, s->d_spart, s->rf_grid,
                                     s->stream, &n_rf);
            e = cudaStreamEndCapture(s->stream, &s->graph);
            if (e == cudaSuccess) e = el;
            s->kernels_per_step = 1 + n_rf;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&s->graph_exec, s->graph, 0);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        destroy_buffers(s);
        delete s;
        return from_cuda(e);
    }
    try {
        s->worker = std::thread(worker_main, s);
    } catch (...) {
        destroy_buffers(s);
        delete s;
        return LYA_ENOMEM;
    }
    *out = s;
    return LYA_OK;
}

lya_status lya_server_submit(lya_server s, lya_field f, const lya_extract_params* p, const int64_t* ids,
                             int64_t n_ids, double target, uint64_t* ticket)
{
    if (!s || !f || !p || !ids || n_ids < 1 || !ticket) return LYA_EINVAL;
    if (!(target > 0.0 && target < 1.0)) return LYA_EINVAL;
    if (p->precision != LYA_PREC_F32_COMPENSATED || p->profile != LYA_PROFILE_SAMPLED ||
        p->exp_method != LYA_EXP_MUFU) return LYA_EINVAL;
    if (f->device != s->device) return LYA_EINVAL;
    if (n_ids > 0x7fffffffLL / f->desc.n_pix) return LYA_EINVAL;
    ReqHost r;
    lya_status st = lya::make_tau_launch(f, p, &r.L);
    if (st != LYA_OK) return st;
    for (int64_t k = 0; k < n_ids; ++k)
        if (ids[k] < 0 || ids[k] >= f->desc.n_skewers) return LYA_EINVAL;
    r.field = f;
    r.Ft = target;
    r.ids.assign(ids, ids + n_ids);
    r.L.err = nullptr;
    const int N = (int)f->desc.n_pix;
    const double ppx = sources_per_pixel(r.L, f);

    std::lock_guard<std::mutex> lk(s->mu);
    if (s->failed != LYA_OK || s->stop) return LYA_ECUDA;
    const int cls = length_class(N);
    const int shift = fit_shift(s, N, r.L.w_max, s->tuned_shift[cls] >= 0 ? s->tuned_shift[cls] : default_shift(N));
    if (shift < 0) return LYA_EINVAL;           // the window does not fit the serving kernel's shared memory
    r.L.err = err_word(s);
    Request q;
    q.ticket = s->next_ticket;
    q.n_rows = n_ids;
    q.n_pix = N;
    q.shift = shift;
    q.row_cost = N * model_ns_per_px(ppx) * s->cost_scale[cls];
    q.task_key = q.row_cost * (double)(1 << shift);
    if (!s->sched->enqueue(q)) return LYA_EBUDGET;
    r.res.n_ids = n_ids;
    r.res.n_pix = N;
    r.res.status = LYA_ENOCONV;
    r.res.t_submit_ns = now_ns();
    f->users.fetch_add(1);
    s->reqs.emplace(q.ticket, std::move(r));
    *ticket = s->next_ticket++;
    ++s->submitted;
    s->cv_work.notify_one();
    return LYA_OK;
}

lya_status lya_server_poll(lya_server s, uint64_t ticket, lya_server_result* out)
{
    if (!s || !out) return LYA_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    return fill_result(s, ticket, out) ? LYA_OK : LYA_EINVAL;
}

lya_status lya_server_wait(lya_server s, uint64_t ticket, double timeout_s, lya_server_result* out)
{
    if (!s || !(timeout_s >= 0.0)) return LYA_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->reqs.count(ticket)) return LYA_EINVAL;
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                              std::chrono::duration<double>(std::min(timeout_s, 1e7)));
    const bool ok = s->cv_done.wait_until(lk, deadline, [&] {
        auto it = s->reqs.find(ticket);
        return it == s->reqs.end() || it->second.res.done;
    });
    if (!fill_result(s, ticket, out)) return LYA_EINVAL;
    return ok ? LYA_OK : LYA_ETIMEDOUT;
}

lya_status lya_server_copy_flux(lya_server s, uint64_t ticket, float* dst, void* stream)
{
    if (!s || !dst) return LYA_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || !it->second.res.done || !it->second.res.flux) return LYA_EINVAL;
    const size_t bytes = sizeof(float) * (size_t)(it->second.res.n_ids * it->second.res.n_pix);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(dst, it->second.res.flux, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the block may be reused once released
    return from_cuda(e);
}

lya_status lya_server_release(lya_server s, uint64_t ticket)
{
    if (!s) return LYA_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return LYA_EINVAL;
    if (!it->second.res.done) return LYA_EBUSY;
    s->sched->release(ticket);
    s->reqs.erase(it);
    s->cv_work.notify_one();                   // memory freed: the queue head may fit now
    return LYA_OK;
}

lya_status lya_server_info(lya_server s, lya_server_info_t* out)
{
    if (!s || !out) return LYA_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->steps = s->steps;
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->n_failed;
    out->arena_used = s->sched->arena().used();
    out->arena_peak = s->sched->arena().peak();
    out->arena_capacity = s->sched->arena().capacity();
    out->slots_in_use = s->sched->slot_ticket_count();
    out->queued = (int)s->sched->queued();
    for (int k = 0; k < kClasses; ++k) out->group_shift[k] = s->tuned_shift[k];
    return LYA_OK;
}

lya_status lya_server_autotune(lya_server s, lya_field f, const lya_extract_params* p, int64_t max_rows,
                               int* shift_out)
{
    if (!s || !f || !p || max_rows < 1) return LYA_EINVAL;
    if (p->precision != LYA_PREC_F32_COMPENSATED || p->profile != LYA_PROFILE_SAMPLED ||
        p->exp_method != LYA_EXP_MUFU || f->device != s->device)
        return LYA_EINVAL;
    TauLaunch L;
    lya_status st = lya::make_tau_launch(f, p, &L);
    if (st != LYA_OK) return st;
    const int N = (int)f->desc.n_pix;
    const int64_t rows = std::min<int64_t>(std::min<int64_t>(max_rows, kMaxItems), f->desc.n_skewers);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->tuning || s->sched->slot_ticket_count() || s->sched->queued()) return LYA_EBUSY;
        if (s->failed != LYA_OK) return LYA_ECUDA;
        s->tuning = true;
    }
    float* tau = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaError_t e = cudaMalloc((void**)&tau, sizeof(float) * (size_t)rows * N);
    if (e == cudaSuccess) e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    int best = -1;
    double best_ns = 0.0;
    std::vector<unsigned char> buf;
    for (int sh = 0; sh <= kMaxShift && e == cudaSuccess; ++sh) {
        if (fit_shift(s, N, L.w_max, sh) != sh) continue;
        // a step of `rows` skewers in tasks of 1 << sh, no root-find
        StepPlan plan;
        plan.tau_slots.push_back(0);
        const int g = 1 << sh;
        for (int64_t r = 0; r < rows; r += g) {
            const int n = (int)std::min<int64_t>(g, rows - r);
            plan.tasks.push_back(StepPlan::Task{0, (int)plan.items.size(), n, sh});
            for (int i = 0; i < n; ++i) plan.items.push_back(StepPlan::Item{0, r + i});
        }
        // lay out directly (the request tables of build_step are not used here)
        unsigned char* b = s->h_step;
        StepHeader* h = reinterpret_cast<StepHeader*>(b);
        std::memset(h, 0, sizeof(StepHeader));
        size_t off = align16(sizeof(StepHeader));
        h->off_slots = off;
        TauLaunch Lt = L;
        Lt.tau_out = tau;
        Lt.err = err_word(s);
        std::memcpy(b + off, &Lt, sizeof(TauLaunch));
        h->n_slots = 1;
        off = align16(off + sizeof(TauLaunch));
        h->off_tasks = off;
        TauTask* T = reinterpret_cast<TauTask*>(b + off);
        for (size_t k = 0; k < plan.tasks.size(); ++k)
            T[k] = TauTask{0, plan.tasks[k].first_item, plan.tasks[k].n_items, sh};
        h->n_tasks = (int)plan.tasks.size();
        off = align16(off + sizeof(TauTask) * plan.tasks.size());
        h->off_items = off;
        TauItem* I = reinterpret_cast<TauItem*>(b + off);
        for (size_t k = 0; k < plan.items.size(); ++k) I[k] = TauItem{(long long)plan.items[k].row, (long long)plan.items[k].row};
        h->n_items = (int)plan.items.size();
        off = align16(off + sizeof(TauItem) * plan.items.size());
        h->off_rf = h->off_units = off;
        const size_t bytes = off;
        float total = 0.f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {       // one warm-up, three timed
            e = cudaMemcpyAsync(s->d_step, s->h_step, bytes, cudaMemcpyHostToDevice, s->stream);
            if (e == cudaSuccess) e = cudaEventRecord(ev0, s->stream);
            if (e == cudaSuccess) e = serve_tau_launch(s->d_step, s->dyn_smem, s->n_sm, s->stream);
            if (e == cudaSuccess) lya::count_launch();
            if (e == cudaSuccess) e = cudaEventRecord(ev1, s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
            if (rep > 0) total += ms;
        }
        const double ns = total / 3.0 * 1e6;
        if (e == cudaSuccess && (best < 0 || ns < best_ns)) {
            best = sh;
            best_ns = ns;
        }
    }
    if (tau) cudaFree(tau);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    int err_h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err_h, err_word(s), sizeof(int), cudaMemcpyDeviceToHost);
    std::lock_guard<std::mutex> lk(s->mu);
    s->tuning = false;
    s->cv_work.notify_one();
    if (e != cudaSuccess) return from_cuda(e);
    if (err_h != 0 || best < 0) return LYA_EINVAL;
    const int cls = length_class(N);
    s->tuned_shift[cls] = best;
    const double model = model_ns_per_px(sources_per_pixel(L, f)) * (double)rows * N;
    s->cost_scale[cls] = best_ns / model;
    if (shift_out) *shift_out = best;
    return LYA_OK;
}

lya_status lya_server_destroy(lya_server s)
{
    if (!s) return LYA_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        fail_all(s, LYA_ECUDA);
    }
    cudaStreamSynchronize(s->stream);
    destroy_buffers(s);
    delete s;
    return LYA_OK;
}

}  // extern "C"
